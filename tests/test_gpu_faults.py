"""Failure paths on the GPU, made on the host side or by a wait that nothing
completes: nothing here faults, traps or hangs the GPU.

- A time-limited device-side wait that runs out records OQR_ERR_TIMEOUT in the
  context's status, and the context stays usable.
- A caller-owned workspace that is too small makes a call return
  OQR_ERR_NO_MEMORY, not allocate; handing the workspace back to the context
  makes the same call succeed.
- A Cholesky breakdown (non-SPD input) returns OQR_ERR_NOT_SPD with its column
  (Algorithm 1 needs G positive definite).
"""
import numpy as np
import pytest

import oracle
from paper_1401_5171_gb300 import inputs

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def env():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1401_5171_gb300 import oqr
    return torch, oqr


def _dev(torch, oqr, x):
    return oqr.colmajor(torch.as_tensor(x).cuda())


def test_timeout_path_leaves_context_usable(env):
    torch, oqr = env
    ctx = oqr.Oqr(0)
    assert ctx.oqr_diag_timeout(1_000_000) == oqr.OQR_ERR_TIMEOUT     # a 1 ms wait that nothing completes
    A, Z = inputs.paper_case(4, 300, 12, 1e3, 1e2, seed=5)
    Q, R, (st, _) = ctx.oqr_cholqr2(_dev(torch, oqr, A), _dev(torch, oqr, Z))
    assert st == oqr.OQR_OK
    Qr, Rr = oracle.oblique_qr(A, Z)
    assert np.linalg.norm(R.cpu().numpy() - Rr) / np.linalg.norm(Rr) <= 1e-12
    ctx.close()


def test_caller_workspace_too_small(env):
    torch, oqr = env
    ctx = oqr.Oqr(0)
    A, Z = inputs.paper_case(4, 400, 16, 1e3, 1e2, seed=6)
    Ad, Zd = _dev(torch, oqr, A), _dev(torch, oqr, Z)
    buf = torch.empty(512, dtype=torch.float64, device="cuda")        # 4 KiB
    ctx.set_workspace(buf.data_ptr(), buf.numel() * 8)
    with pytest.raises(oqr.OqrError) as e:
        ctx.oqr_cholqr2(Ad, Zd, opts=oqr.make_opts(prec=oqr.OQR_TC2, final_prec=oqr.OQR_FP64_TC))
    assert e.value.status == oqr.OQR_ERR_NO_MEMORY
    ctx.set_workspace(0, 0)                                            # the context allocates again
    Q, R, (st, _) = ctx.oqr_cholqr2(Ad, Zd, opts=oqr.make_opts(prec=oqr.OQR_TC2, final_prec=oqr.OQR_FP64_TC))
    assert st == oqr.OQR_OK
    ctx.close()


def test_not_spd_reports_column(env):
    torch, oqr = env
    ctx = oqr.Oqr(0)
    A = np.eye(80)
    A[5, 5] = -2.0                                                     # indefinite: G breaks at column 6
    Z = np.eye(80, 8)
    Q, R, (st, info) = ctx.oqr_cholqr2(_dev(torch, oqr, A), _dev(torch, oqr, Z), raise_on_error=False)
    assert st == oqr.OQR_ERR_NOT_SPD and info.info == 6
    ctx.close()
