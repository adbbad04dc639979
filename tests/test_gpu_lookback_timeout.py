"""The bounded look-back of the onesweep sort gives up and reports DARB_ERR_TIMEOUT instead of
hanging.  A test build of the library (DARB_TEST_HOOKS, DARB_SPIN_LIMIT = 1024 polls, so the
wait lasts well under a millisecond) runs one pass whose partition 0 is never processed, so the
one CTA's look-back waits on a status that nothing publishes.  The call must come back with the
timeout in the status word and the stream completed; the device stays usable afterwards."""
import ctypes

import pytest
import torch

pytestmark = [pytest.mark.gpu,
              pytest.mark.skipif(not torch.cuda.is_available(), reason="needs a CUDA GPU")]

DARB_ERR_TIMEOUT = 5


@pytest.fixture(scope="module")
def hooks():
    from paper_2501_12369_gb300 import build
    path = build.build_variant("test_hooks", ["-DDARB_TEST_HOOKS=1", "-DDARB_SPIN_LIMIT=1024"])
    L = ctypes.CDLL(path)
    L.darb_test_lookback_timeout_bytes.restype = ctypes.c_size_t
    L.darb_test_lookback_timeout_bytes.argtypes = []
    L.darb_test_lookback_timeout.restype = ctypes.c_int32
    L.darb_test_lookback_timeout.argtypes = [ctypes.c_void_p, ctypes.c_size_t, ctypes.POINTER(ctypes.c_uint32),
                                             ctypes.c_void_p]
    return L


def test_lookback_wait_runs_out_and_reports_timeout(hooks):
    nbytes = hooks.darb_test_lookback_timeout_bytes()
    ws = torch.empty(nbytes, dtype=torch.uint8, device="cuda")
    stream = torch.cuda.current_stream()
    for _ in range(2):  # twice: the first timeout leaves nothing behind that the second trips over
        status = ctypes.c_uint32(0)
        rc = hooks.darb_test_lookback_timeout(ctypes.c_void_p(ws.data_ptr()), nbytes, ctypes.byref(status),
                                              ctypes.c_void_p(stream.cuda_stream))
        assert rc == 0, f"the call itself failed: {rc}"
        assert status.value == DARB_ERR_TIMEOUT
    torch.cuda.synchronize()
    x = torch.arange(1000, device="cuda", dtype=torch.float32)
    assert float(x.sum()) == 499500.0  # the context is intact


def test_normal_library_has_no_test_hook():
    from paper_2501_12369_gb300 import build, darb
    build.build()
    assert not hasattr(darb.lib(), "darb_test_lookback_timeout")
