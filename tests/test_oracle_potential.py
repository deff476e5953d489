"""Pins of the oracle's potential-solve RF source (sigma |grad V|^2 of Eq.
2675-eq1_Linte with div(sigma grad V) = 0): a series resistor, the discrete
power balance (Tellegen), the maximum principle, symmetry, and the power
normalisation."""
import numpy as np

import oracle
import phantoms as ph


def test_two_material_resistor():
    nx, h = 20, 1e-3
    s1, s2 = 0.2, 0.8
    sig = np.where(np.arange(nx) < 9, s1, s2).astype(np.float64).reshape(1, 1, nx)
    sf = oracle.harmonic_faces(sig)
    el = np.zeros((1, 1, nx), bool)
    gr = np.zeros((1, 1, nx), bool)
    el[..., 0] = True
    gr[..., -1] = True
    V = oracle.potential_solve(sf, el, gr)[0, 0]
    s = sig[0, 0]
    sfx = 2 * s[:-1] * s[1:] / (s[:-1] + s[1:])
    J = 1.0 / np.sum(1.0 / sfx)                  # current x h per unit area (V = 1 across)
    Vx = 1.0 - J * np.concatenate([[0.0], np.cumsum(1.0 / sfx)])
    assert np.allclose(V, Vx, rtol=0, atol=1e-12)
    q = oracle.joule(V.reshape(1, 1, nx), sf, h)[0, 0]
    fd = sfx * np.diff(Vx) ** 2                  # sigma_f dV^2 per face
    qx = np.zeros(nx)
    qx[:-1] += fd / (2 * h * h)
    qx[1:] += fd / (2 * h * h)
    assert np.allclose(q, qx, rtol=1e-12, atol=0)


def test_tellegen_power_balance_and_maximum_principle():
    rng = np.random.default_rng(5)
    shape = (11, 13, 12)
    h = 0.7e-3
    sig = rng.uniform(0.1, 1.0, size=shape)
    sf = oracle.harmonic_faces(sig)
    z, y, x = np.meshgrid(*(np.arange(n) for n in shape), indexing="ij")
    gr = (x == 0) | (y == 0) | (z == 0) | (x == shape[2] - 1) | (y == shape[1] - 1) | (z == shape[0] - 1)
    el = ((x - 6) ** 2 + (y - 6) ** 2 + (z - 5) ** 2 <= 4) & ~gr
    V = oracle.potential_solve(sf, el, gr)
    assert V.min() >= -1e-14 and V.max() <= 1 + 1e-14
    q = oracle.joule(V, sf, h)
    # current leaving the electrode: sum over its faces of sigma_f (V_e - V_nb) h
    I = 0.0
    for d in range(6):
        nb, ok = oracle._shift(V, d)
        I += np.sum(np.where(el & ok, sf[d] * (1.0 - nb) * h, 0.0))
    assert np.sum(q) * h ** 3 == __import__("pytest").approx(1.0 * I, rel=1e-10)


def test_symmetry_of_a_centred_needle():
    n, h = 21, 1e-3
    c = (n - 1) / 2 * h
    case = ph.homogeneous_case(n=n, h=h)
    case.needle = ph.Needle(kind=ph.STRAIGHT, tip=(c, c, c + 4 * h), active_len=8 * h, power=5.0)
    case.source = "potential"
    m = oracle.setup(case, "f64")
    V, q, s = oracle.potential_source(case, m)
    assert np.allclose(V, V[:, :, ::-1], atol=1e-12)
    assert np.allclose(V, V[:, ::-1, :], atol=1e-12)
    assert np.allclose(V, np.swapaxes(V, 1, 2), atol=1e-12)
    # the normalised source delivers exactly the needle power to the free voxels
    P = np.sum(s * m.rhoc) * h ** 3 / case.dt
    assert P == __import__("pytest").approx(5.0, rel=1e-12)
    assert np.array_equal(m.s, s)
