"""Section 3.3 subwarp reduction benchmark kernel: parity of all three
implementations with the oracle's butterfly definition (integer data, so
the comparison is exact)."""
import numpy as np
import pytest

import oracle as O
from gpu_util import dev, host

pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("S", [1, 2, 4, 8, 16, 32])
@pytest.mark.parametrize("impl", [0, 1, 2])
@pytest.mark.parametrize("dt", ["f64", "f32"])
@pytest.mark.parametrize("loops", [0, 1, 3])
def test_subwarp_reduce_matches_oracle(gko, S, impl, dt, loops):
    G = gko
    rng = np.random.default_rng(S + 7 * impl + 100 * loops)
    d = rng.integers(-9, 10, 1024).astype(np.float64)
    t = dev(d) if dt == "f64" else dev(d, np.float32)
    G.gko_bench_subwarp_reduce(S, impl, t, loops)
    np.testing.assert_array_equal(host(t).astype(np.float64), O.subwarp_reduce(d, S, loops))


def test_subwarp_reduce_rejects_bad_arguments(gko):
    G = gko
    t = dev(np.zeros(256))
    for S, impl in [(3, 0), (64, 0), (4, 3)]:
        with pytest.raises(G.GkoError):
            G.gko_bench_subwarp_reduce(S, impl, t, 1)
    with pytest.raises(G.GkoError):
        G.gko_bench_subwarp_reduce(4, 0, dev(np.zeros(100)), 1)
