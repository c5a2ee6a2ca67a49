"""Failure detection on the GPU without a fault: a bounded wait on a barrier
that nothing completes gives up within its limit, the time-out reaches the
host as GKO_TIMEOUT through the device error word, and the context keeps
working (an SpMV afterwards matches the oracle)."""
import time

import numpy as np
import pytest

from gpu_util import check_spmv_f64, dev, host
from paper_2006_14290_gb300 import inputs as I

pytestmark = pytest.mark.gpu


def test_bounded_wait_times_out_and_context_survives(gko):
    G = gko
    G.gko_device_status()  # clean start
    t0 = time.perf_counter()
    assert G.gko_diag_bounded_wait(20_000_000)  # about 10 ms at 2 GHz
    assert time.perf_counter() - t0 < 5.0
    with pytest.raises(G.GkoError) as e:
        G.gko_device_status()
    assert e.value.status == G.TIMEOUT
    G.gko_device_status()  # the word was cleared by the read
    A = I.stencil3d_27pt(12)
    M = G.from_csr(A)
    x = np.random.default_rng(0).uniform(-1, 1, A.n_cols)
    yd = dev(np.zeros(A.n_rows))
    G.gko_spmv(1.0, M, dev(x), 0.0, yd)
    check_spmv_f64(host(yd), A, x, 1.0, 0.0, None)
    G.gko_device_status()


def test_bounded_wait_rejects_bad_limits(gko):
    G = gko
    for bad in (0, -5, 2**33):
        with pytest.raises(G.GkoError) as e:
            G.gko_diag_bounded_wait(bad)
        assert e.value.status == G.INVALID_ARG
