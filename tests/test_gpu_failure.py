"""Failure detection on the device without a fault: a bounded wait that runs
out reports FDTD_ETIMEOUT through the status word and leaves the context
usable; a non-finite state is reported as FDTD_EUNSTABLE (test_gpu_parity)."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("no CUDA device", allow_module_level=True)

import workloads
import test_gpu_parity as tp

pytestmark = pytest.mark.gpu


def test_bounded_wait_reports_timeout_and_context_survives():
    w = workloads.cavity_60(120)
    ctx, _ = tp.gpu_context([w])
    assert ctx.selftest_timeout() == -7          # FDTD_ETIMEOUT
    assert ctx.selftest_timeout() == -7          # reported again, not stuck
    g = tp.gpu_run(ctx, [w], 120)                # the context still runs
    ref_ctx, _ = tp.gpu_context([w])
    np.testing.assert_array_equal(g, tp.gpu_run(ref_ctx, [w], 120))
