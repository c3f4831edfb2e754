"""bte_init_maxwellian_static: the initial-state fill for callers that cannot allocate device memory.

It must give what bte_init_maxwellian gives, through the C ABI, on consecutive calls (the static
scratch array is shared and keeps the previous call's contents), with a normal handle and with a
host-only handle (one that holds no device memory), and it must refuse to be recorded into a CUDA
graph (its coefficient copy reads a host buffer that does not outlive the call)."""
import ctypes as C

import numpy as np
import pytest

from paper_2502_16555_gb300 import workloads as W
from tests._lib import ensure_built

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _built():
    ensure_built()
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")


def _ref_and_static(s_ref, h_static, lib, ne, Te):
    """Fill once through bte_init_maxwellian and once through the static-scratch entry point."""
    from paper_2502_16555_gb300 import bte
    F_ref = s_ref.empty_state()
    s_ref.init_maxwellian(F_ref, ne, Te)
    F_st = torch.full_like(F_ref, float("nan"))
    st = lib.bte_init_maxwellian_static(h_static, C.c_void_p(F_st.data_ptr()), C.c_void_p(ne.data_ptr()), float(Te))
    assert st == bte.OK, lib.bte_last_error(h_static)
    torch.cuda.synchronize()
    return F_ref.cpu().numpy(), F_st.cpu().numpy()


def _check(F_ref, F_st):
    scale = np.abs(F_ref).max()
    assert np.all(np.isfinite(F_st))
    assert np.max(np.abs(F_st - F_ref)) <= 1e-14 * scale


def test_static_fill_matches_init_maxwellian_two_calls():
    from paper_2502_16555_gb300 import bte
    lib = bte.load()
    cfg = W.scaled(W.SMALL, nx=11, nr=24, ntheta=6)
    s = bte.Solver(cfg, precision="fp64")
    rng = np.random.default_rng(7)
    ne1 = torch.tensor(1e15 * rng.uniform(0.1, 1.0, cfg["nx"]), dtype=torch.float64, device="cuda")
    ne2 = torch.tensor(3e14 * rng.uniform(0.1, 1.0, cfg["nx"]), dtype=torch.float64, device="cuda")
    _check(*_ref_and_static(s, s.h, lib, ne1, 2.0))
    _check(*_ref_and_static(s, s.h, lib, ne2, 0.7))   # second call: other Te, other n_e


def test_static_fill_with_host_only_handle():
    from paper_2502_16555_gb300 import bte
    lib = bte.load()
    cfg = W.scaled(W.SMALL, nx=9, nr=40, ntheta=4)
    s = bte.Solver(cfg, precision="fp64")
    s_host = bte.Solver(cfg, host_only=True)
    ne = torch.linspace(1e13, 1e15, cfg["nx"], dtype=torch.float64, device="cuda")
    _check(*_ref_and_static(s, s_host.h, lib, ne, 1.5))
    _check(*_ref_and_static(s, s_host.h, lib, ne, 4.0))


def test_static_fill_refuses_stream_capture():
    """While the handle's stream is capturing, the call returns BTE_ESTATE and records nothing: the
    replayed graph leaves the state buffer as it was."""
    from paper_2502_16555_gb300 import bte
    lib = bte.load()
    cfg = W.scaled(W.SMALL, nx=7, nr=12, ntheta=4)
    stream = torch.cuda.Stream()
    s = bte.Solver(cfg, precision="fp64", stream=stream)
    ne = torch.full((cfg["nx"],), 1e15, dtype=torch.float64, device="cuda")
    F = torch.empty((cfg["nx"], cfg["ntheta"], cfg["nr"]), dtype=torch.float64, device="cuda")
    ptr = lambda t: C.c_void_p(t.data_ptr())
    # the first call on the device, outside any capture
    assert lib.bte_init_maxwellian_static(s.h, ptr(F), ptr(ne), 2.0) == bte.OK
    torch.cuda.synchronize()
    F.fill_(7.0)
    counter = torch.zeros(1, dtype=torch.float64, device="cuda")
    torch.cuda.synchronize()
    g = torch.cuda.CUDAGraph()
    with torch.cuda.stream(stream):
        g.capture_begin()
        counter.add_(1.0)
        st = lib.bte_init_maxwellian_static(s.h, ptr(F), ptr(ne), 2.0)
        g.capture_end()
    assert st == bte.ESTATE, lib.bte_last_error(s.h)
    g.replay()
    torch.cuda.synchronize()
    assert counter.item() == 1.0
    assert torch.all(F == 7.0)
    # usable again once the capture has ended
    assert lib.bte_init_maxwellian_static(s.h, ptr(F), ptr(ne), 2.0) == bte.OK
    torch.cuda.synchronize()
    assert torch.all(torch.isfinite(F)) and not torch.all(F == 7.0)
