"""Host logic of the exact 2D projection, without a device: the tables that
stc_dct_tables builds (and stc_create_problem uploads) against scipy's
orthonormal DCT-II and the closed-form eigenvalues of the cell-centred
Neumann Laplacian, and the four-product solve assembled from them against the
oracle's sparse direct Poisson solve (test infrastructure: oracle/)."""
import numpy as np
import pytest
import scipy.fft

from oracle import mac, projection
from paper_1608_01102_gb300 import stc


@pytest.mark.parametrize("nx,ny", [(8, 8), (12, 8), (10, 6), (32, 24)])
def test_tables_are_the_orthonormal_dct_and_the_laplacian_spectrum(nx, ny):
    t = stc.dct_tables(nx, ny)
    for n, C, CT in ((nx, t["Cx"], t["CxT"]), (ny, t["Cy"], t["CyT"])):
        ref = scipy.fft.dct(np.eye(n), type=2, norm="ortho", axis=0)   # column i = DCT of e_i
        np.testing.assert_allclose(C, ref, atol=1e-14)
        np.testing.assert_array_equal(CT, C.T)
        np.testing.assert_allclose(C @ C.T, np.eye(n), atol=1e-13)
    h = 1.0 / nx
    kx, ky = np.arange(nx), np.arange(ny)
    lam = -(4 / h ** 2) * (np.sin(np.pi * ky / (2 * ny))[:, None] ** 2 + np.sin(np.pi * kx / (2 * nx))[None, :] ** 2)
    assert t["inv_lam"][0, 0] == 0.0
    m = np.ones_like(lam, dtype=bool)
    m[0, 0] = False
    np.testing.assert_allclose(t["inv_lam"][m], 1.0 / lam[m], rtol=1e-14)


@pytest.mark.parametrize("nx,ny", [(8, 8), (12, 8), (16, 10)])
def test_four_products_solve_the_neumann_poisson_problem(nx, ny):
    t = stc.dct_tables(nx, ny)
    g = mac.Grid(nx, ny, 1.0 / nx)
    rng = np.random.default_rng(9)
    b = rng.standard_normal(g.C)
    b -= b.mean()
    B = b.reshape(ny, nx)
    phi = t["CyT"] @ ((t["Cy"] @ B @ t["CxT"]) * t["inv_lam"]) @ t["Cx"]
    ref = projection.poisson_neumann(g, b).reshape(ny, nx)
    np.testing.assert_allclose(phi - phi.mean(), ref, atol=1e-11 * np.max(np.abs(ref)))


def test_bad_arguments_are_rejected():
    lib = stc.load()
    out = np.zeros(3)
    assert lib.stc_dct_tables(0, 4, out.ctypes.data_as(stc.P_double), out.size) != 0
    assert lib.stc_dct_tables(4, 4, None, 100) != 0
    assert lib.stc_dct_tables(4, 4, out.ctypes.data_as(stc.P_double), out.size) != 0   # needs 2*16+2*16+16
