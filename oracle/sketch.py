"""Sparse sign embedding S (Sec. 2.1, Eq. 3), generated column by column.

S = (1/sqrt(zeta)) [s_1 ... s_n] is d x n (d is called ``s`` here, as in the
GPU library).  Every column s_j holds zeta nonzeros equal to +-1 at row
positions chosen uniformly at random; the signs are Rademacher.

Readings of the paper (it does not fix the generator, Sec. 2.1 and App. A):
* rows are drawn WITHOUT replacement, so every column has exactly zeta
  distinct rows and ||S e_j||_2 = 1 exactly;
* the random stream of column j is Philox4x32-10 with key (seed lo, seed hi)
  and counters (j, block, 0, 0), block = 0, 1, 2, ...; each output block gives
  four 32-bit words and every word two 16-bit chunks, low half first;
* a chunk c yields a candidate row v = c & 0x7FFF and a sign bit c >> 15;
  the candidate is rejected if v >= 32768 - (32768 mod s) (so that v mod s is
  exactly uniform) or if row = v mod s was already chosen for this column;
  an accepted chunk contributes the entry (row, -1 if the sign bit is set
  else +1);
* at most MAX_BLOCKS blocks are drawn per column; running out is an error.
Constraints: 1 <= zeta <= min(s, 32) and s <= 32768.
"""
import numpy as np

from .philox import philox4x32_10

MAX_BLOCKS = 64


def sketch_columns(n, s, zeta, seed, cols=None):
    """Rows (int64, len(cols) x zeta) and signs (+-1.0) of the selected columns.

    Entries of a column are listed in the order they were accepted.
    """
    if not (1 <= zeta <= min(s, 32)) or s > 32768:
        raise ValueError("need 1 <= zeta <= min(s, 32) and s <= 32768")
    cols = np.arange(n, dtype=np.int64) if cols is None else np.asarray(cols, dtype=np.int64)
    m = cols.size
    rows = np.full((m, zeta), -1, dtype=np.int64)
    signs = np.zeros((m, zeta))
    count = np.zeros(m, dtype=np.int64)
    lim = 32768 - (32768 % s)
    k0 = seed & 0xFFFFFFFF
    k1 = (seed >> 32) & 0xFFFFFFFF
    for block in range(MAX_BLOCKS):
        active = np.nonzero(count < zeta)[0]
        if active.size == 0:
            break
        words = philox4x32_10(cols[active], block, 0, 0, k0, k1)
        for w in words:
            for half in (0, 1):
                chunk = ((w >> np.uint64(16 * half)) & np.uint64(0xFFFF)).astype(np.int64)
                v = chunk & 0x7FFF
                neg = (chunk >> 15) == 1
                row = v % s
                # candidate of each still-active column
                fresh = ~np.any(rows[active] == row[:, None], axis=1)
                take = (count[active] < zeta) & (v < lim) & fresh
                idx = active[take]
                rows[idx, count[idx]] = row[take]
                signs[idx, count[idx]] = np.where(neg[take], -1.0, 1.0)
                count[idx] += 1
    if np.any(count < zeta):
        raise RuntimeError("sparse sign generator ran out of random blocks")
    return rows, signs


class SparseSign:
    """The d x n embedding, materialized once per run (Sec. 2.1, App. A)."""

    def __init__(self, n, s, zeta, seed):
        self.n, self.s, self.zeta, self.seed = n, s, zeta, seed
        self.rows, self.signs = sketch_columns(n, s, zeta, seed)

    def apply(self, v):
        """S v for a vector v (n,) or every column of V (n, k): FP64 sums in
        column order, each entry scaled by 1/sqrt(zeta)."""
        v = np.asarray(v, dtype=np.float64)
        scale = 1.0 / np.sqrt(self.zeta)
        if v.ndim == 1:
            contrib = (self.signs * scale) * v[:, None]
            return np.bincount(self.rows.ravel(), weights=contrib.ravel(), minlength=self.s)
        return np.stack([self.apply(v[:, i]) for i in range(v.shape[1])], axis=1)

    def dense(self):
        """S as a dense s x n array (tiny n only)."""
        D = np.zeros((self.s, self.n))
        for q in range(self.zeta):
            D[self.rows[:, q], np.arange(self.n)] += self.signs[:, q] / np.sqrt(self.zeta)
        return D
