"""m2c_step_host, the host-resident time-stepping loop in one call per step (upload from pinned
host arrays, step, download back; a call's upload overlapping the previous call's download one
state component at a time): the same state bit for bit as the device-resident run and as the
separate upload / step / download calls, over calls on the same arrays, after a switch to other
arrays, and after other work on the context in between (which ends the overlap)."""
import numpy as np
import pytest

from paper_2508_16387_gb300 import workloads as WL

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def env():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no GPU")
    from paper_2508_16387_gb300 import m2c as M
    from paper_2508_16387_gb300 import runner as RN
    M.lib()
    return torch, M, RN


@pytest.mark.parametrize("prec", [0, 1])
def test_host_loop_equals_device_run(env, prec):
    torch, M, RN = env
    s = WL.shock_bubble(n=40, radius=0.18, centre=(0.47, 0.52, 0.5), p_shock=8e8, steps=30)
    ref = RN.grid_for(s, prec)
    sep = RN.grid_for(s, prec)
    g = RN.grid_for(s, prec)
    shape_W, shape_p = tuple(g.W.shape), tuple(g.phi.shape)
    Wh = torch.empty(shape_W, dtype=torch.float64, pin_memory=True)
    ph = torch.empty(shape_p, dtype=torch.float64, pin_memory=True)
    Ws = torch.empty(shape_W, dtype=torch.float64, pin_memory=True)
    pss = torch.empty(shape_p, dtype=torch.float64, pin_memory=True)
    g.download(Wh, ph)
    sep.download(Ws, pss)
    W2 = torch.empty(shape_W, dtype=torch.float64, pin_memory=True)
    p2 = torch.empty(shape_p, dtype=torch.float64, pin_memory=True)
    for k in range(12):
        ref.step(1)
        sep.upload(Ws, pss)
        sep.step(1)
        sep.download(Ws, pss)
        if k == 5:
            # other arrays for two calls (no overlap with the previous call's copies)
            g.sync()
            W2.copy_(Wh)
            p2.copy_(ph)
            g.step_host(W2, p2, 1)
            g.step_host(W2, p2, 1)
            g.sync()
            Wh.copy_(W2)
            ph.copy_(p2)
        elif k == 6:
            continue
        elif k == 9:
            # other work on the context in between: the state query ends the overlap
            g.step_host(Wh, ph, 1)
            g.stats()
            g.prims()
        else:
            g.step_host(Wh, ph, 1)
    t_ref, n_ref = ref.sync()
    t_g, n_g = g.sync()
    assert n_ref == n_g == 12 and t_ref == t_g
    assert np.array_equal(Wh.numpy(), ref.W.cpu().numpy())
    assert np.array_equal(ph.numpy(), ref.phi.cpu().numpy())
    assert np.array_equal(Ws.numpy(), ref.W.cpu().numpy())


def test_host_loop_rejects_bad_arguments(env):
    torch, M, RN = env
    s = WL.shock_bubble(n=16, steps=2)
    g = RN.grid_for(s, 1)
    Wh = torch.empty(tuple(g.W.shape), dtype=torch.float64, pin_memory=True)
    ph = torch.empty(tuple(g.phi.shape), dtype=torch.float64, pin_memory=True)
    with pytest.raises(M.M2CError):
        g.step_host(Wh, ph, -1)
    assert M.lib().m2c_step_host(g.ctx, None, None, 1) == M.M2C_EINVAL
