"""Failure handling on the GPU without a fault: a pipeline barrier that nothing
completes makes the tcgen05 kernel's bounded wait give up after about a second,
report through its error flag and leave the context usable (include/dot_selftest.h)."""
import ctypes

import pytest

from gpu_util import ensure_built

pytestmark = pytest.mark.gpu


def run(lib, inject):
    secs = ctypes.c_double(0.0)
    flag = ctypes.c_int(-1)
    rc = lib.dot_selftest_pipeline_timeout(int(inject), ctypes.byref(secs), ctypes.byref(flag))
    return rc, secs.value, flag.value


def test_wait_that_never_completes_reports_and_the_context_survives():
    lib = ensure_built()
    rc, secs, flag = run(lib, False)
    assert rc == 0 and flag == 0
    rc, secs, flag = run(lib, True)
    assert rc == 0 and flag == 1
    assert 0.5 < secs < 10.0            # the one-second limit of the bounded waits
    rc, secs, flag = run(lib, False)    # the same process and device go on working
    assert rc == 0 and flag == 0 and secs < 0.5
