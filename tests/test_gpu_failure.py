"""Failure detection on the GPU without a fault: a bounded wait that runs out
reports SSSGS_STATUS_TIMEOUT in the status word, the context stays usable, and
the host side turns the status into an error."""
import time

import pytest
import torch

import scenegen as sg
from paper_2408_12282_gb300 import binding as B
from paper_2408_12282_gb300 import pipeline as PL

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _lib(gpu_lib):
    return gpu_lib


def test_bounded_wait_times_out_and_the_context_stays_usable():
    st = torch.zeros(1, dtype=torch.int32, device="cuda")
    t0 = time.perf_counter()
    B.selftest_wait_timeout(st, 2_000_000)          # about 1 ms of SM clock cycles, nothing arrives
    torch.cuda.synchronize()
    dt = time.perf_counter() - t0
    assert int(st.item()) & B.STATUS_TIMEOUT
    assert dt < 5.0
    wl = sg.make_workload("c1", N=256, res=32)
    r = PL.renderer_for_workload(wl)
    r.fit_capacity()
    r.forward()
    torch.cuda.synchronize()
    r.check_status()
    assert torch.isfinite(r.img).all()
    r.status.fill_(B.STATUS_TIMEOUT)                 # what a timed-out tensor-core kernel leaves behind
    with pytest.raises(B.SSSGSError):
        r.check_status()
    with pytest.raises(B.SSSGSError):
        B.selftest_wait_timeout(st, 0)               # out-of-range limit: refused on the host
