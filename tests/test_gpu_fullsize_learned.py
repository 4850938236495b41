"""Full-size parity of the learned Hamiltonian at the 10-million-atom graphene
configuration (2500 x 1000 rectangular cells, 0.1 A Gaussian disorder,
learned H stored as FP32 SELL), in the launch configuration of the
benchmark (neighbour list with 16-wide slices, descriptors, tcgen05 forward,
symmetrisation and onsite sums at N = 1e7).

The oracle cannot build the whole 1e7-atom learned H, so the check is on
sampled rows S.  H_ij of a row i needs the outputs of both directed edges
i -> j and j -> i (the symmetrisation after Eq. 2), hence the node features
v of i and of every neighbour j (Eq. 2), hence the neighbour lists of
S and N(S).  These all lie within 2 r_cut of S, so the oracle takes the
atoms within 2 r_cut + 1 A of a sampled row (minimum image, a brute-force
scan of all 1e7 positions per sampled row) and runs its brute force of the
neighbour definition on that subset: distances do not depend on which
other atoms are present, so the lists are those of the full system.

Per sampled row the oracle then forms the radial descriptors (Eq. 2), the
FP64 forward of the 32-64-64-2 network with BF16-rounded weights and
BF16-rounded normalised inputs (the precision the tensor-core forward takes
its operands in), H_ij = (y(i->j) + y(j->i)) / 2 and eps_i = eps0 +
sum_j y_on(i->j).  Bars: neighbour indices bit-exact; hoppings and onsite
terms within 1e-2 relative L2 (a BF16 operand differing by one unit in the
last place moves an output by about 4e-3 of its size)."""
import numpy as np
import pytest
import torch

from oracle import descriptors as ode
from oracle import mlp as omlp
from oracle import neighbors as onb
from paper_2509_06525_gb300 import synth

pytestmark = [pytest.mark.gpu, pytest.mark.slow]


@pytest.fixture(scope="module")
def g():
    from paper_2509_06525_gb300 import build, gputb
    build.build()
    return gputb


def _bf16(a):
    return torch.tensor(np.asarray(a, np.float32)).bfloat16().double().numpy()


def _near(pos, box, pbc, centre, radius):
    """Indices of atoms within `radius` of `centre` (per-component minimum
    image of an orthorhombic box)."""
    d = pos - centre
    lengths = np.diag(box)
    for k in range(3):
        if pbc[k]:
            d[:, k] -= lengths[k] * np.rint(d[:, k] / lengths[k])
    return np.nonzero(np.sum(d * d, axis=1) < radius * radius)[0]


def test_learned_hamiltonian_10M_atoms(g):
    w = synth.WORKLOADS["graphene-10M-learned"]
    s = synth.graphene_rect(w["nx"], w["ny"], w["sigma"], w["seed"])
    p = synth.teacher_graphene()
    assert s.n == 10_000_000 and onb.is_orthorhombic(s.box)
    rcut = p.rcut

    # the sampled rows and the oracle's neighbour lists of S and N(S)
    rng = np.random.default_rng(11)
    rows = np.unique(np.concatenate([[0, 1, w["nx"] * 4 - 1, s.n // 2, s.n - 1],
                                     rng.choice(s.n, 27, replace=False)]))
    subset = np.unique(np.concatenate([_near(s.positions, s.box, s.pbc, s.positions[i], 2 * rcut + 1.0)
                                       for i in rows]))
    local = {int(a): k for k, a in enumerate(subset)}
    lists = {}
    sub_pos = s.positions[subset]

    def fill(atoms):
        need = [a for a in atoms if a not in lists]
        for a, (idx, dv) in zip(need, onb.neighbors_of_rows(sub_pos, s.box, s.pbc, rcut, [local[a] for a in need])):
            lists[a] = (subset[idx], dv)

    fill([int(i) for i in rows])
    fill(sorted({int(j) for i in rows for j in lists[int(i)][0]}))

    # oracle descriptors: C per directed edge, v per atom (Eq. 2)
    cm = synth.descriptor_mixing("identity")
    cm64 = cm.astype(np.float64)
    C, v = {}, {}
    for a, (idx, dv) in lists.items():
        r = np.sqrt(np.sum(dv * dv, axis=1))
        C[a] = ode.mixed_descriptor(r, np.full(idx.size, s.species[a]), s.species[idx], cm64, rcut)
        v[a] = C[a].sum(axis=0)
    x, owner = [], []
    for i in rows:
        i = int(i)
        for e, j in enumerate(lists[i][0]):
            j = int(j)
            back = int(np.searchsorted(lists[j][0], i))
            assert lists[j][0][back] == i
            cij, cji = C[i][e], C[j][back]
            x.append(np.concatenate([cij, v[i], v[j], cij * (v[i] + v[j])]))
            x.append(np.concatenate([cji, v[j], v[i], cji * (v[j] + v[i])]))
            owner.append((i, j))
    x = np.asarray(x)
    mean, std = x.mean(0), x.std(0)
    assert np.all(std > 1e-3)

    # device: the launch configuration of the benchmark's learned step
    seed = 21
    model = g.MLPModel(synth.init_mlp(seed), cm, np.zeros(3))
    model.set_normalisation(torch.tensor(mean, device="cuda"), torch.tensor(std, device="cuda"))
    pos = torch.tensor(s.positions, device="cuda")
    spc = torch.tensor(s.species, device="cuda")
    nb = g.build_neighbors(pos, s.box, s.pbc, rcut, r_count=p.r_count, max_width=16)
    assert nb.n == s.n
    vd = g.compute_descriptors(pos, spc, s.box, s.pbc, rcut, nb, model.cmix)
    H = g.build_hamiltonian(pos, spc, s.box, s.pbc, rcut, nb, model, v=vd, dtype=torch.float32, with_diag=True)
    torch.cuda.synchronize()

    # neighbour indices bit-exact on the sampled rows and their neighbours
    sp_, cnt = nb.slice_ptr.cpu().numpy(), nb.cnt.cpu().numpy()

    def slots(i):
        k, lane = divmod(int(i), 32)
        return sp_[k] + lane + 32 * np.arange(cnt[i])

    col = nb.col
    for a, (idx, _) in lists.items():
        np.testing.assert_array_equal(col[torch.tensor(slots(a), device="cuda")].cpu().numpy(), idx)

    # node features: the device's FP32 sums against the oracle's
    atoms = sorted(lists)
    v_dev = vd[torch.tensor(atoms, device="cuda")].cpu().numpy().astype(np.float64)
    v_ref = np.stack([v[a] for a in atoms])
    np.testing.assert_allclose(v_dev, v_ref, rtol=2e-5, atol=2e-5)

    # oracle forward, symmetrisation and onsite terms
    params = {k: np.asarray(val, np.float64) for k, val in synth.init_mlp(seed).items()}
    for k in ("W1", "W2", "W3"):
        params[k] = _bf16(params[k])
    y, _ = omlp.forward(params, _bf16((x - mean) / std), np.zeros(32), np.ones(32))
    hop_ref = 0.5 * (y[0::2, 0] + y[1::2, 0])
    on_ref = {int(i): 0.0 for i in rows}
    for (i, _), yo in zip(owner, y[0::2, 1]):
        on_ref[i] += yo

    e_dev = np.concatenate([slots(i) for i in rows])
    hop = H.val[torch.tensor(e_dev, device="cuda")].cpu().numpy().astype(np.float64)
    rel = float(np.linalg.norm(hop - hop_ref) / np.linalg.norm(hop_ref))
    assert rel <= 1e-2, f"sampled hoppings differ from the oracle (rel L2 {rel})"
    on = H.diag[torch.tensor(rows, device="cuda")].cpu().numpy().astype(np.float64)
    on_r = np.array([on_ref[int(i)] for i in rows])
    rel_on = float(np.linalg.norm(on - on_r) / np.linalg.norm(on_r))
    assert rel_on <= 1e-2, f"sampled onsite terms differ from the oracle (rel L2 {rel_on})"
    # H is symmetric: the stored (j, i) entry equals the (i, j) one bit for bit
    for i in rows[:8]:
        for e, j in zip(slots(i), lists[int(i)][0]):
            back = slots(j)[int(np.searchsorted(lists[int(j)][0], int(i)))]
            assert float(H.val[int(e)]) == float(H.val[int(back)])
