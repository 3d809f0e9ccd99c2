"""Failure reporting and resumption, exercised without faulting or hanging the GPU:
a non-finite objective ends a solve with NCS_ERR_DIVERGED; the tensor-core
convolution's bounded waits, made to run out by the test-only switch, end the call with
NCS_ERR_TIMEOUT and leave the context usable; and a solver state copied to the host and
back resumes with bitwise-identical iterates (the kernels are deterministic)."""
import numpy as np
import pytest

import synth
from helpers import oproj

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


def test_nan_in_data_reports_divergence():
    import paper_1810_13100_gb300 as ncs
    N, na, nd = 48, 60, 70
    b = synth.ct_problem(1, N, na, nd, 6, 0.01, oproj(N, na, nd))["b"].ravel().copy()
    b[123] = np.nan
    plan = ncs.Plan(N, na, nd, 0.05, 0.01, power_max_iter=2)
    x = torch.zeros(N * N, device="cuda")
    with pytest.raises(ncs.NCSError) as e:
        plan.solve(torch.from_numpy(b).cuda(), x, tol=1e-4, max_iter=50)
    assert e.value.code == ncs.binding.NCS_ERR_DIVERGED
    # the plan still works on good data
    b[123] = 0.0
    rep = plan.solve(torch.from_numpy(b).cuda(), x.zero_(), tol=0.0, max_iter=20)
    assert np.isfinite(rep["f"])
    plan.close()


def test_tensor_core_wait_timeout_is_reported_and_recoverable():
    import paper_1810_13100_gb300 as ncs
    H = 32
    net = ncs.UNet(H, H, levels=2, base=16, seed=2)
    x = torch.rand(H * H, device="cuda", generator=torch.Generator(device="cuda").manual_seed(0))
    y_ok = net.forward(x).clone()
    net.inject_wait_timeout()
    with pytest.raises(ncs.NCSError) as e:
        net.forward(x)
    assert e.value.code == ncs.binding.NCS_ERR_TIMEOUT
    y_again = net.forward(x)
    assert torch.equal(y_again, y_ok)
    net.close()


def test_state_round_trip_through_host_resumes_bitwise():
    import paper_1810_13100_gb300 as ncs
    N, na, nd = 64, 90, 92
    b = torch.from_numpy(synth.ct_problem(2, N, na, nd, 10, 0.01, oproj(N, na, nd))["b"].ravel()).cuda()
    plan = ncs.Plan(N, na, nd, 0.01, 0.01, tv="aniso")
    z = lambda k: torch.zeros(k, device="cuda")
    x, u, v = z(N * N), z(na * nd), z(2 * N * N)
    plan.step(x, u, v, None, b, n_iter=30)
    x2, u2, v2 = z(N * N), z(na * nd), z(2 * N * N)
    plan.step(x2, u2, v2, None, b, n_iter=12)
    saved = [t.cpu().numpy().copy() for t in (x2, u2, v2)]
    plan.close()
    plan2 = ncs.Plan(N, na, nd, 0.01, 0.01, tv="aniso")
    x3, u3, v3 = (torch.from_numpy(a).cuda() for a in saved)
    plan2.step(x3, u3, v3, None, b, n_iter=18)
    torch.cuda.synchronize()
    assert torch.equal(x3, x) and torch.equal(u3, u) and torch.equal(v3, v)
    plan2.close()
