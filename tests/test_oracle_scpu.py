"""The streaming Gram update on the host cores (oracle/stream_cpu.c, the timed
streaming CPU baseline; Sec. 3.1, Eq. 12a-b) against the definition: after
every push, the physical G over the slots in use equals the brute-force Gram
of the ring's contents (numpy integer products: exact), through the window's
ramp-up and several wraps, with n spanning several 32768-position blocks and
a ragged tail. FP32 windows: FP64 sums within 1e-12 relative."""

import numpy as np
import pytest

from oracle import native


def _ring_gram_i64(ring, used):
    R = ring[:used].astype(np.int64)
    return R @ R.T


@pytest.mark.parametrize("n,m", [(3 * 32768 + 1234, 6), (1000, 1), (32768, 4)])
def test_streaming_u8_equals_brute_force(n, m):
    rng = np.random.default_rng(n + m)
    sc = native.StreamingCPU(n, m, "u8")
    for t in range(2 * m + 3):
        x = rng.integers(0, 256, n, dtype=np.uint8)
        if t == 1:
            x[:] = 255                                   # the largest products
        s = sc.push(x)
        assert s == t % m
        assert np.array_equal(sc.ring[s], x)
        used = min(t + 1, m)
        assert np.array_equal(sc.G[:used, :used], _ring_gram_i64(sc.ring, used)), t


def test_streaming_f32_equals_fp64_dots():
    n, m = 70001, 5
    rng = np.random.default_rng(7)
    sc = native.StreamingCPU(n, m, "f32")
    for t in range(2 * m + 1):
        x = rng.standard_normal(n).astype(np.float32)
        sc.push(x)
        used = min(t + 1, m)
        R = sc.ring[:used].astype(np.float64)
        ref = R @ R.T
        assert np.abs(sc.G[:used, :used] - ref).max() <= 1e-12 * np.abs(ref).max(), t


def test_streaming_rejects_bad_arguments():
    L = native.lib()
    ring = np.zeros((4, 100), dtype=np.uint8)
    G = np.zeros((4, 4), dtype=np.int64)
    x = np.zeros(100, dtype=np.uint8)
    args = dict(pitch=100, n=100, m=4, used=2, s_new=1)
    assert L.scpu_push_u8(ring.ctypes.data, 100, 100, 4, 2, 1, x.ctypes.data, G.ctypes.data) == 0
    for bad in ({"s_new": 2}, {"used": 5}, {"used": 0}, {"m": 300}, {"pitch": 99}):
        a = dict(args, **bad)
        assert L.scpu_push_u8(ring.ctypes.data, a["pitch"], a["n"], a["m"], a["used"], a["s_new"],
                              x.ctypes.data, G.ctypes.data) == -1, bad
    with pytest.raises(ValueError):
        native.StreamingCPU(10, 3, "u8").push(np.zeros(11, dtype=np.uint8))
