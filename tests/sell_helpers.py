"""Test-side helpers: pack an oracle CSR matrix into the SELL-32 layout of
include/gputb.h (host NumPy), and pick up the CUDA binding."""
import numpy as np

SLICE = 32


def csr_to_sell(indptr, indices, values, n):
    """(slice_ptr int64, col int32, val float64) with padding col = i, val = 0.

    Slice k holds rows 32k .. 32k + 31 in `width_k` slots, slot-major: element
    s of row i sits at slice_ptr[k] + (i mod 32) + 32 s.  Lanes past the last
    row (n not a multiple of 32) keep col = 0, val = 0."""
    indptr = np.asarray(indptr, np.int64)
    indices = np.asarray(indices)
    values = np.asarray(values, np.float64)
    counts = np.diff(indptr)
    n_slices = (n + SLICE - 1) // SLICE
    padded = np.zeros(n_slices * SLICE, np.int64)
    padded[:n] = counts
    widths = padded.reshape(n_slices, SLICE).max(axis=1)
    slice_ptr = np.zeros(n_slices + 1, np.int64)
    slice_ptr[1:] = np.cumsum(widths * SLICE)
    total = int(slice_ptr[-1])
    col = np.zeros(total, np.int32)
    val = np.zeros(total, np.float64)
    if total == 0:
        return slice_ptr, col, val
    pos = np.arange(total, dtype=np.int64)
    k = np.repeat(np.arange(n_slices, dtype=np.int64), widths * SLICE)
    off = pos - slice_ptr[k]
    row = k * SLICE + off % SLICE
    s = off // SLICE
    real = row < n
    pos, row, s = pos[real], row[real], s[real]
    col[pos] = row
    used = s < counts[row]
    src = indptr[row[used]] + s[used]
    col[pos[used]] = indices[src]
    val[pos[used]] = values[src]
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
