"""Seeded input generator: stream definition and recipe statistics (CPU)."""
import math

import numpy as np
import pytest

import synth

M64 = (1 << 64) - 1


def philox4x64_10(ctr, key):
    """Philox4x64-10 round function (Salmon et al., SC'11), plain Python ints."""
    c, k = list(ctr), list(key)
    for _ in range(10):
        p0 = 0xD2E7470EE14C6C93 * c[0]
        p1 = 0xCA5A826395121157 * c[2]
        c = [(p1 >> 64) ^ c[1] ^ k[0], p1 & M64, (p0 >> 64) ^ c[3] ^ k[1], p0 & M64]
        k = [(k[0] + 0x9E3779B97F4A7C15) & M64, (k[1] + 0xBB67AE8584CAA73B) & M64]
    return c


def test_raw_stream_is_philox_counter_layout():
    raw = synth.raw_stream(7, 9, 12)
    for r in range(12):
        blk = philox4x64_10([r // 4 + 1, 0, 0, 0], [7, 9])
        assert int(raw[r]) == blk[r % 4]


def test_normals_moments():
    e = synth.normals(3, synth.STREAM_X, 400000)
    assert abs(e.mean()) < 0.01
    assert e.var() == pytest.approx(1.0, abs=0.01)
    assert np.mean(np.abs(e) > 1.96) == pytest.approx(0.05, abs=0.003)


def test_ar1_design_correlation():
    X = synth.ar1_design(4000, 6, 0.7, 1)
    C = np.corrcoef(X.T)
    for d in range(1, 4):
        assert C[0, d] == pytest.approx(0.7 ** d, abs=0.05)
    assert X.var(axis=0).mean() == pytest.approx(1.0, abs=0.05)


def test_response_snr_and_labels():
    X, y = synth.make_problem_cpu(synth.WORKLOADS["ls_500x1000_f64"])
    s = synth.signal_from_design(X, 10)
    noise = y - s
    assert np.dot(s, s) / np.dot(noise, noise) == pytest.approx(5.0, rel=0.2)
    w = synth.WORKLOADS["logistic_20000x50000_f32"]
    _, yl = synth.make_problem_cpu(w, n=300, p=200)
    assert set(np.unique(yl)) <= {-1.0, 1.0}


def test_support_and_fixings():
    assert list(synth.support(50000, 50)[:3]) == [0, 1000, 2000]
    f = synth.node_fixings(10000, 0, 5, 40, 19, k=20)
    assert np.sum(f < 0) <= 40 and np.sum(f > 0) <= 19
    assert np.array_equal(f, synth.node_fixings(10000, 0, 5, 40, 19, k=20))


def test_paper_sweep_workloads():
    # Sec. 5.2's root-relaxation sweep: n = p, rho 0.5, k 10, M 2, lambda2 1
    for p in (1000, 2000, 4000, 8000, 16000):
        for loss in ("ls", "logistic"):
            w = synth.WORKLOADS[f"paper_{loss}_{p}x{p}_f32"]
            assert (w.n, w.p, w.rho, w.k, w.M, w.lambda2, w.loss) == (p, p, 0.5, 10, 2.0, 1.0, loss)
    X, y = synth.make_problem_cpu(synth.WORKLOADS["paper_logistic_1000x1000_f32"])
    assert X.shape == (1000, 1000) and set(np.unique(y)) <= {-1.0, 1.0}
