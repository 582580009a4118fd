"""Pins for the synthetic problem generators against closed forms."""
import numpy as np
import pytest

from paper_1712_07297_gb300 import inputs as I


def _lap_eigs(shape):
    lam = [2.0 - 2.0 * np.cos(np.arange(1, s + 1) * np.pi / (s + 1)) for s in shape]
    grids = np.meshgrid(*lam, indexing="ij")
    return np.sort(sum(grids).reshape(-1))


@pytest.mark.parametrize("shape", [(16,), (7, 9), (4, 5, 6)])
def test_laplacian_spectrum_closed_form(shape):
    # eigenvalues of the Dirichlet Laplacian: sum_d 4 sin^2(i_d pi / (2 (n_d + 1)))
    p = I.poisson(shape)
    A = p.dense()
    np.testing.assert_allclose(np.linalg.eigvalsh(A), _lap_eigs(shape), atol=1e-12)


def test_laplacian_sine_eigenvector():
    shape = (5, 6, 7)
    p = I.poisson(shape)
    idx = (2, 3, 1)
    x = p.coords
    v = np.ones(p.n)
    lam = 0.0
    for d, s in enumerate(shape):
        v *= np.sin((idx[d]) * np.pi * (x[:, d] + 1) / (s + 1))
        lam += 2 - 2 * np.cos(idx[d] * np.pi / (s + 1))
    np.testing.assert_allclose(p.scipy() @ v, lam * v, atol=1e-12)


def test_csr_layout():
    p = I.poisson((3, 4, 5))
    assert p.rowptr.dtype == np.int64 and p.col.dtype == np.int32 and p.val.dtype == np.float64
    assert p.rowptr[0] == 0 and p.rowptr[-1] == p.nnz == len(p.col)
    for i in range(p.n):
        c = p.col[p.rowptr[i]:p.rowptr[i + 1]]
        assert np.all(np.diff(c) > 0) and i in c
    # 7-point stencil: interior row has 7 entries
    assert np.max(np.diff(p.rowptr)) == 7


def test_convection_diffusion_m_matrix():
    p = I.convection_diffusion((4, 4, 4), 10.0)
    A = p.dense()
    assert not np.allclose(A, A.T)
    assert np.all(np.diag(A) == 36.0)
    off = A - np.diag(np.diag(A))
    assert np.all(off <= 0)
    # interior row sums vanish (consistent upwind discretisation), others >= 0
    assert np.all(A.sum(axis=1) >= -1e-12)
    assert set(np.unique(off[off != 0])) == {-11.0, -1.0}
    # M-matrix: inverse is elementwise nonnegative
    assert np.all(np.linalg.inv(A) >= -1e-14)


def test_vc_diffusion_harmonic_faces():
    p = I.vc_diffusion((3, 3, 3), seed=7)
    A = p.dense()
    np.testing.assert_allclose(A, A.T)
    # row sums are the Dirichlet boundary faces' own coefficients
    rng = np.random.default_rng(7)
    a = 10.0 ** rng.uniform(-3, 3, size=27)
    nb = np.zeros(27)
    for c in range(27):
        x, y, z = c % 3, (c // 3) % 3, c // 9
        nb[c] = sum(1 for q in (x, y, z) for e in (0, 2) if q == e) * a[c]
    np.testing.assert_allclose(A.sum(axis=1), nb, rtol=1e-12, atol=1e-12 * np.abs(A).max())
    # face coefficient between cells 0 and 1 is the harmonic mean
    np.testing.assert_allclose(-A[0, 1], 2 * a[0] * a[1] / (a[0] + a[1]), rtol=1e-14)


def test_high_contrast_two_values():
    p = I.high_contrast((12, 12, 12), seed=3)
    A = p.dense()
    offv = -A[(A != 0) & ~np.eye(p.n, dtype=bool)]
    # harmonic means of {1e2, 1e-2}: 1e2, 1e-2 or 2e-2/(1+1e-4)
    allowed = np.array([1e2, 1e-2, 2 * 1e2 * 1e-2 / (1e2 + 1e-2)])
    assert np.all(np.min(np.abs(offv[:, None] - allowed[None, :]) / allowed, axis=1) < 1e-12)


def test_rhs_seeded():
    b1 = I.rhs(100, 3, seed=5)
    b2 = I.rhs(100, 3, seed=5)
    assert b1.shape == (3, 100) and b1.flags.c_contiguous
    np.testing.assert_array_equal(b1, b2)
    assert b1.min() >= -1 and b1.max() <= 1
