"""GB300-native GPUTB hot path: neighbour search, descriptors, learned or
teacher tight-binding Hamiltonian in sliced-ELL form, spectral bounds and
the KPM Chebyshev recursion for the density of states; the VAC
conductivity, the s, p, d Slater-Koster model, and the environment-network
model with band-energy training (``bands``).

The compute path is the CUDA library ``libgputb.so`` behind the C ABI in
``include/gputb.h``; ``paper_2509_06525_gb300.gputb`` is its thin Python
binding.  This ``__init__`` imports nothing so that ``synth`` (seeded
inputs) can be used without loading the library.
"""
