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


@pytest.mark.parametrize("dt", ["f64", "f32"])
def test_fma_probe_runs_the_stated_recurrence(gko, dt):
    """gko_bench_fma: 8 chains v <- v*a + b per thread (a = 1 - 2^-10,
    b = 2^-10, chain c from seed + c/8), the sum stored; checked against
    the same recurrence on the host (fused vs unfused rounding: a
    tolerance of a few units in the last place per step)."""
    G = gko
    rng = np.random.default_rng(5)
    seeds = rng.uniform(-4, 4, 512)
    loops = 37
    npt = np.float64 if dt == "f64" else np.float32
    t = dev(seeds) if dt == "f64" else dev(seeds, np.float32)
    G.gko_bench_fma(t, loops)
    s0 = seeds.astype(npt)
    a, b = npt(0.9990234375), npt(0.0009765625)
    want = np.zeros(512, np.float64)
    for c in range(8):
        v = (s0 + npt(c) * npt(0.125)).astype(npt)
        for _ in range(loops):
            v = (v * a + b).astype(npt)
        want += v.astype(np.float64)
    got = host(t).astype(np.float64)
    tol = 1e-12 if dt == "f64" else 2e-4
    np.testing.assert_allclose(got, want, rtol=tol, atol=tol)
    with pytest.raises(G.GkoError):
        G.gko_bench_fma(dev(np.zeros(100)), 1)


@pytest.mark.parametrize("dt", ["f64", "f32"])
def test_gather_probe_xors_the_stated_elements(gko, dt):
    """gko_bench_gather: thread t keeps states 8t + c, steps them by the
    stated linear congruence and xors element (s >> (32 - k)) of x into its
    accumulator; the host replays the same integer recurrence (bit-exact)."""
    G = gko
    k, n, loops = 12, 512, 5
    npt, ut = (np.float64, np.uint64) if dt == "f64" else (np.float32, np.uint32)
    xh = np.random.default_rng(7).uniform(-1, 1, 1 << k).astype(npt)
    x = dev(xh) if dt == "f64" else dev(xh, np.float32)
    out = dev(np.zeros(n)) if dt == "f64" else dev(np.zeros(n), np.float32)
    G.gko_bench_gather(x, out, loops)
    bits = xh.view(ut)
    st = (np.arange(n, dtype=np.uint64)[:, None] * 8 + np.arange(8, dtype=np.uint64)[None, :]) & 0xFFFFFFFF
    acc = np.zeros(n, ut)
    for _ in range(loops):
        st = (st * 1664525 + 1013904223) & 0xFFFFFFFF
        idx = (st >> (32 - k)) & ((1 << k) - 1)
        for c in range(8):
            acc ^= bits[idx[:, c]]
    np.testing.assert_array_equal(host(out).view(ut), acc)
    with pytest.raises(ValueError):
        G.gko_bench_gather(dev(np.zeros(100)), out, 1)
