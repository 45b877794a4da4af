"""Checks of the seeded input generators (links and Z4 noise)."""

import numpy as np

from paper_1405_4524_gb300 import inputs


def test_links_are_su3():
    U = inputs.make_links((4, 4, 2, 6), 0.25, 1)
    UdU = np.conj(np.swapaxes(U, -1, -2)) @ U
    assert np.allclose(UdU, np.eye(3), atol=1e-14)
    assert np.allclose(np.linalg.det(U), 1.0, atol=1e-14)


def test_link_generator_normalisation():
    # H traceless Hermitian with E[tr H^2] = 9 - 1 = 8
    rng = np.random.default_rng(0)
    h = inputs._traceless_hermitian(rng.standard_normal((200000, 3, 3, 2)))
    assert np.allclose(h, np.conj(np.swapaxes(h, -1, -2)))
    assert np.allclose(np.trace(h, axis1=-2, axis2=-1), 0)
    m = np.mean(np.real(np.trace(h @ h, axis1=-2, axis2=-1)))
    assert abs(m - 8.0) < 0.05


def test_links_are_deterministic_and_smooth():
    a = inputs.make_links((2, 2, 2, 4), 0.25, 5)
    b = inputs.make_links((2, 2, 2, 4), 0.25, 5)
    assert np.array_equal(a, b)
    # eps = 0.25: mean Re tr U / 3 close to 1 - eps^2 * 8 / 6
    U = inputs.make_links((8, 8, 8, 8), 0.25, 6)
    m = np.mean(np.real(np.trace(U, axis1=-2, axis2=-1))) / 3
    assert abs(m - (1 - 0.25 ** 2 * 8 / 6)) < 0.01


def test_z4_noise():
    eta = inputs.make_z4((4, 4, 4, 8), 8, 10)
    assert np.allclose(np.abs(eta), 1.0)
    vals = set(np.round(eta.ravel()[:1000], 12).tolist())
    assert vals <= {1, 1j, -1, -1j}
    assert abs(np.mean(eta)) < 0.02
    # E[eta_i eta_j^*] = delta_ij; E[eta^2] = 0 for Z4
    flat = eta.reshape(8, -1)
    gram = flat @ flat.conj().T / flat.shape[1]
    assert np.allclose(gram, np.eye(8), atol=0.05)
    assert abs(np.mean(flat ** 2)) < 0.02


def test_time_dilution():
    eta = inputs.make_z4((2, 2, 2, 8), 3, 4, tslices=[0, 5, 9])
    for k, t in enumerate([0, 5, 1]):
        nz = np.nonzero(np.abs(eta[k]).sum(axis=(1, 2, 3, 4, 5)))[0]
        assert nz.tolist() == [t]
