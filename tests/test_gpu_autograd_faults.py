"""torch.autograd.gradcheck through the autograd shim (FP64 form, tiny inputs exact in float32),
and the bounded waits: a CTA that never receives its tile makes the call report DBIE_ETIMEOUT
after the wait limit, and the context keeps working."""
import ctypes

import numpy as np
import pytest

from test_gpu_eval import random_mag, random_points

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def dbie():
    import paper_1306_1122_gb300 as d
    return d


def test_gradcheck_through_dbie_apply(dbie):
    """dbie_apply (B0, lambda) -> B: gradcheck's central differences against the adjoint and
    dB/dlambda.  B0 on multiples of 1/16 and a difference step of 1/64 stay exact in float32 (B is
    linear in B0); lambda on multiples of 2^-12 with a step of 2^-10 likewise."""
    rng = np.random.default_rng(3)
    ny, nx, n = 4, 5, 4
    B0 = torch.from_numpy(np.round(rng.normal(0, 20, (ny, nx, 3)) * 16) / 16).cuda()
    f = dbie.DBIEField(B0[..., 0].float(), B0[..., 1].float(), B0[..., 2].float())
    xyz = torch.from_numpy(np.stack([rng.uniform(0, 4, n), rng.uniform(0, 3, n),
                                     rng.uniform(0.8, 3, n)], 1).astype(np.float32)).cuda()
    lam = torch.from_numpy(np.round(rng.uniform(-0.4, 0.4, (n, 3)) * 4096) / 4096).cuda()
    opt = dbie.Options(precision=1)
    B0.requires_grad_(True)
    lam.requires_grad_(True)
    fn = lambda b0, l: dbie.dbie_apply(f, b0, l, xyz, opt)
    # the lambda columns carry the O(eps^2) truncation of central differences (~1e-6 against a
    # Jacobian of order 1): absolute tolerance 1e-5
    assert torch.autograd.gradcheck(fn, (B0, lam), eps=2.0 ** -10, atol=1e-5, rtol=1e-4)
    f.close()


def test_bounded_wait_timeout_is_reported_and_context_survives(dbie, monkeypatch):
    import paper_1306_1122_gb300._native as N
    mag = random_mag(40, 30, 5)
    xyz, lam = random_points(mag, 500, 6)
    h = N.dbie_create(mag.nx, mag.ny, mag.x0, mag.y0, mag.hx, mag.hy, mag.dA,
                      *(c.ctypes.data_as(ctypes.c_void_p) for c in (mag.Bx, mag.By, mag.Bz)),
                      N.DBIE_MEM_HOST, None)
    P = lambda a: a.ctypes.data_as(ctypes.c_void_p)
    B_ok = np.zeros((500, 3))
    N.dbie_eval(h, 500, P(xyz), P(lam), None, N.DBIE_MEM_HOST, P(B_ok), None, None, None, None)
    monkeypatch.setenv("DBIE_FAULT_INJECT", "1")
    B_bad = np.zeros((500, 3))
    with pytest.raises(N.DBIEError) as e:
        N.dbie_eval(h, 500, P(xyz), P(lam), None, N.DBIE_MEM_HOST, P(B_bad), None, None, None,
                    None)
    assert e.value.status == N.DBIE_ETIMEOUT
    monkeypatch.delenv("DBIE_FAULT_INJECT")
    B_again = np.zeros((500, 3))
    N.dbie_eval(h, 500, P(xyz), P(lam), None, N.DBIE_MEM_HOST, P(B_again), None, None, None, None)
    N.dbie_destroy(h)
    assert np.array_equal(B_again, B_ok)
    assert torch.cuda.is_available() and torch.zeros(1).cuda().item() == 0.0
