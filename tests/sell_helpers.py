"""Test-side helpers: pack an oracle CSR matrix into the SELL-32 layout of
include/gputb.h (host NumPy), and pick up the CUDA binding."""
import numpy as np

SLICE = 32


def csr_to_sell(indptr, indices, values, n):
    """(slice_ptr int64, col int32, val float64) with padding col = i, val = 0."""
    indptr = np.asarray(indptr)
    counts = np.diff(indptr)
    n_slices = (n + SLICE - 1) // SLICE
    widths = np.zeros(n_slices, np.int64)
    for k in range(n_slices):
        widths[k] = counts[k * SLICE:(k + 1) * SLICE].max(initial=0)
    slice_ptr = np.zeros(n_slices + 1, np.int64)
    slice_ptr[1:] = np.cumsum(widths * SLICE)
    col = np.zeros(slice_ptr[-1], np.int32)
    val = np.zeros(slice_ptr[-1], np.float64)
    for i in range(n):
        k, lane = divmod(i, SLICE)
        base = slice_ptr[k] + lane
        row = slice(indptr[i], indptr[i + 1])
        m = counts[i]
        pos = base + SLICE * np.arange(widths[k])
        col[pos] = i
        col[pos[:m]] = indices[row]
        val[pos[:m]] = values[row]
    return slice_ptr, col, val


def sell_matrix(indptr, indices, values, onsite, n, dtype, device="cuda"):
    import torch
    from paper_2509_06525_gb300 import gputb
    sp, col, val = csr_to_sell(indptr, indices, values, n)
    diag = None
    if onsite is not None and np.any(onsite != 0):
        diag = torch.tensor(onsite, dtype=dtype, device=device)
    return gputb.SellMatrix(n, torch.tensor(sp, device=device), torch.tensor(col, device=device),
                            torch.tensor(val, dtype=dtype, device=device), diag)
