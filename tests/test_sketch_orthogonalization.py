"""The GPU's randomized Gram-Schmidt step orthogonalizes the sketch of each
product against the window's sketches by classical Gram-Schmidt applied
twice, where Algorithm 1 prints a modified Gram-Schmidt loop.  On CPU
(numpy, float64): the two give the same coefficients up to rounding, and
twice-applied classical Gram-Schmidt keeps the sketched basis orthonormal to
rounding also when the new vector lies nearly in the span of the window,
where one modified pass does not ("twice is enough")."""
import numpy as np


def mgs(Q, p):
    r = np.zeros(Q.shape[1])
    p = p.copy()
    for i in range(Q.shape[1]):
        r[i] = Q[:, i] @ p
        p -= r[i] * Q[:, i]
    return r, p


def cgs2(Q, p):
    r1 = Q.T @ p
    p1 = p - Q @ r1
    r2 = Q.T @ p1
    return r1 + r2, p1 - Q @ r2


def sketched_basis(rng, s, k):
    Q, _ = np.linalg.qr(rng.standard_normal((s, k)))
    return Q


def test_cgs2_and_mgs_coefficients_agree():
    rng = np.random.default_rng(21)
    for s, k in ((160, 2), (160, 40), (320, 40)):
        Q = sketched_basis(rng, s, k)
        p = rng.standard_normal(s)
        r_m, q_m = mgs(Q, p)
        r_c, q_c = cgs2(Q, p)
        assert np.abs(r_m - r_c).max() <= 1e-14 * np.linalg.norm(p)
        assert np.linalg.norm(q_m - q_c) <= 1e-14 * np.linalg.norm(p)


def test_cgs2_keeps_orthogonality_for_nearly_dependent_vectors():
    """A product nearly in the span of the window: one pass, classical or
    modified, leaves the normalized result with components along the window
    that grow like u / eps; the second classical pass removes them."""
    rng = np.random.default_rng(22)
    s, k = 160, 40
    for eps in (1e-4, 1e-8, 1e-12):
        Q = sketched_basis(rng, s, k)
        p = Q @ rng.standard_normal(k) + eps * rng.standard_normal(s)
        _, q = cgs2(Q, p)
        assert np.abs(Q.T @ (q / np.linalg.norm(q))).max() <= 1e-15
        for one_pass in (mgs(Q, p)[1], p - Q @ (Q.T @ p)):
            loss = np.abs(Q.T @ (one_pass / np.linalg.norm(one_pass))).max()
            assert loss <= 1e-15 / eps
            if eps <= 1e-8:
                assert loss > 1e-11
