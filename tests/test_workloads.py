"""The seeded synthetic inputs at the sizes the benchmark and the parity tests
quote (CPU; the generators hold none of the method's arithmetic)."""
import numpy as np

import workloads as W


def test_headline_operator_at_full_size():
    """3D upwind convection-diffusion, 128^3 interior nodes, beta = 50 on
    every axis: n = 2,097,152, nnz = 7 n - 6 * 128^2, three distinct values,
    each exact in float32 (the float32 value copy is lossless)."""
    A = W.convdiff3d(128)
    assert (A.n, A.nnz) == (2_097_152, 14_581_760)
    vals = np.unique(A.val)
    assert set(vals.tolist()) == {119196.0, -16641.0, -23091.0}
    assert np.array_equal(vals.astype(np.float32).astype(np.float64), vals)
    assert A.row_ptr[-1] == A.nnz and np.all(np.diff(A.row_ptr) >= 4)
    assert np.diff(A.row_ptr).max() == 7


def test_fem_size_from_its_pattern():
    """The P1 Kuhn stiffness matrix couples each interior node along seven
    edge directions (both signs) and to itself; on (cells - 1)^3 interior
    nodes that gives n + 2 (3 (N-1) N^2 + 3 (N-1)^2 N + (N-1)^3) entries:
    59,690,347 at 160^3 cells, and the generator agrees at a small size."""
    def nnz(N):
        return N ** 3 + 2 * (3 * (N - 1) * N ** 2 + 3 * (N - 1) ** 2 * N + (N - 1) ** 3)

    F = W.fem_p1_kuhn(10, 1.0, 3)
    assert (F.n, F.nnz) == (9 ** 3, nnz(9))
    assert (159 ** 3, nnz(159)) == (4_019_679, 59_690_347)
