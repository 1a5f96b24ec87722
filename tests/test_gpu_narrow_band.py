"""The narrow-band level set (Sec. 4.4; Reading R38, the local level set of Peng et
al.) on the GPU against the oracle: the stage residual <= 1e-11, FP64 runs
<= 1e-9 for the density, the momentum vector and the energy with an identical
sign pattern of phi and the level set itself <= 1e-9 of the tube radius, the
mixed path <= 1e-4 relative L1 of rho and p."""
import numpy as np
import pytest

from oracle import oracle as O
from paper_2508_16387_gb300 import workloads as WL
from tests.metrics import conserved_errors as rel_err

pytestmark = pytest.mark.gpu

TOL = 1e-9
BAND = dict(band_beta=3.0, band_gamma=6.0)


@pytest.fixture(scope="module")
def m2c():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no GPU")
    from paper_2508_16387_gb300 import m2c as M
    M.lib()
    return M


def test_band_residual_matches_oracle(m2c):
    n = (40, 22, 18)
    P, phi = WL.random_state(n, seed=19, two_phase=True)
    bc = (0, 0, 1, 1, 0, 0)
    eos = (WL.WATER_SG, WL.AIR_PG)
    g_or = O.Grid(n=n, h=1.0 / n[0], eos=tuple(O.EOS(*e) for e in eos), bc=bc, band_beta=2.0, band_gamma=4.0)
    R_ref, L_ref, _ = O.residual(g_or, O.prims_to_cons(g_or, P, phi), phi)
    g = m2c.Grid(n, 1.0 / n[0], bc, eos, options=dict(band_beta=2.0, band_gamma=4.0))
    g.set_prims(P, phi)
    R, L = g.residual()
    R, L = R.cpu().numpy(), L.cpu().numpy()
    assert max(rel_err(R, R_ref)) < 1e-11
    assert np.abs(L - L_ref).max() <= 1e-11 * max(np.abs(L_ref).max(), 1.0)
    assert np.count_nonzero(L_ref == 0.0) > 0 and np.count_nonzero(L == 0.0) == np.count_nonzero(L_ref == 0.0)


@pytest.mark.parametrize("reinit", [(10, 5), (1, 3)])
@pytest.mark.parametrize("precision", [0, 1])
def test_shock_bubble_with_a_band_matches_oracle(m2c, reinit, precision):
    s = WL.shock_bubble(n=40, radius=0.18, centre=(0.47, 0.52, 0.5), p_shock=8e8, steps=80)
    g_or = O.Grid(n=s.n, h=s.h, eos=tuple(O.EOS(*e) for e in s.eos), bc=s.bc, reinit_every=reinit[0],
                  reinit_iters=reinit[1], **BAND)
    amb = s.prims_by_region[s.shock[1]]
    r1, u1, _ = O.shock_state(O.EOS(*s.eos[0]), (amb[0], amb[1], amb[4]), s.shock[0])
    ref = O.run(g_or, O.prims_to_cons(g_or, s.prims((r1, u1)), s.phi), s.phi, 80)
    g = m2c.Grid(s.n, s.h, s.bc, s.eos, precision=precision, reinit_every=reinit[0], reinit_iters=reinit[1],
                 options=BAND)
    r1g, u1g, _ = m2c.m2c_shock_state(s.eos[0], (amb[0], amb[1], amb[4]), s.shock[0])
    g.set_prims(s.prims((r1g, u1g)), s.phi)
    g.step(80)
    g.sync()
    phi = g.phi.cpu().numpy()
    assert np.abs(phi).max() <= 6.0 * s.h
    if precision == 0:
        assert max(rel_err(g.W.cpu().numpy(), ref.W)) <= TOL
        assert np.array_equal(phi < 0, ref.phi < 0)
        assert np.abs(phi - ref.phi).max() <= TOL * 6.0 * s.h
    else:
        Pg = O.cons_to_prims(g_or, g.W.cpu().numpy(), phi)
        Pr = O.cons_to_prims(g_or, ref.W, ref.phi)
        for v in (0, 4):
            A = Pg[v].reshape(10, 4, 10, 4, 10, 4).mean(axis=(1, 3, 5))
            B = Pr[v].reshape(10, 4, 10, 4, 10, 4).mean(axis=(1, 3, 5))
            assert np.abs(A - B).sum() / np.abs(B).sum() <= 1e-4, v


def test_translating_sphere_with_a_band_matches_oracle(m2c):
    """The oracle pin's translating sphere (one gas, uniform flow, periodic box, reinitialised
    every step) on the GPU."""
    n = 32
    h = 1.0 / n
    c = (np.arange(n) + 0.5) * h
    z, y, x = np.meshgrid(c, c, c, indexing="ij")
    phi = np.sqrt((x - 0.4) ** 2 + (y - 0.4) ** 2 + (z - 0.5) ** 2) - 0.25
    P = np.zeros((5,) + phi.shape)
    P[0] = 1.0
    P[1] = P[2] = 300.0 / np.sqrt(2.0)
    P[4] = 1e5
    eos = (WL.AIR_PG, WL.AIR_PG)
    g_or = O.Grid(n=(n, n, n), h=h, eos=tuple(O.EOS(*e) for e in eos), bc=(1,) * 6, reinit_every=1,
                  reinit_iters=5, **BAND)
    ref = O.run(g_or, O.prims_to_cons(g_or, P, phi), phi, 100)
    g = m2c.Grid((n, n, n), h, (1,) * 6, eos, reinit_every=1, reinit_iters=5, options=BAND)
    g.set_prims(P, phi)
    g.step(100)
    g.sync()
    out = g.phi.cpu().numpy()
    assert np.array_equal(out < 0, ref.phi < 0)
    assert np.abs(out - ref.phi).max() <= TOL * 6.0 * h
