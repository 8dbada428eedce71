"""The seeded input generator: determinism and the recipe's statistics (CPU)."""
import numpy as np

from paper_2207_12244_gb300 import synth


def test_keyframe_recipe():
    a = synth.make_keyframe(256, 192, 0)
    b = synth.make_keyframe(256, 192, 0)
    for p, q in zip(a.cnn_planes + (a.mu_s, a.var_s), b.cnn_planes + (b.mu_s, b.var_s)):
        assert p.dtype == np.float32 and p.shape == (192, 256) and p.flags.c_contiguous
        assert np.array_equal(p, q)
    D = np.exp(a.log_depth_true)
    assert D.min() >= 0.5 - 1e-9 and D.max() <= 5.0 + 1e-9
    assert abs((a.var_s > 0).mean() - 0.2) < 1e-3
    assert np.all(a.var_n >= 0.05 ** 2 * 0.999) and np.all(a.var_n <= 0.3 ** 2 * 1.001)
    assert np.all(a.var_gx[:, :-1] >= 1e-4 * 0.999) and np.all(a.var_gx[:, :-1] <= 1e-2 * 1.001)
    assert 0.5 <= np.exp(a.scale_log_true) <= 2.0
    assert abs(np.std(a.mu_n - a.log_depth_true) - 0.1) < 0.005
    m = a.var_s > 0
    z = (a.mu_s[m] + a.scale_log_true - a.log_depth_true[m]) / np.sqrt(a.var_s[m])
    assert abs(z.std() - 1.0) < 0.03
    c = synth.make_keyframe(256, 192, 1)
    assert not np.array_equal(a.mu_n, c.mu_n)


def test_sequence_recipe():
    kf, mus, vs = synth.make_sequence(64, 48, 3, n_frames=20)
    fr = (vs > 0).reshape(20, -1).mean(axis=1)
    assert abs(fr[0] - 0.05) < 0.01 and abs(fr[-1] - 0.40) < 0.01
    assert np.all(np.diff(fr) >= 0)
    m0 = vs[0] > 0
    assert np.all(vs[-1][m0] <= vs[0][m0])  # fusion only shrinks variances
    assert np.all((vs[5] > 0) <= (vs[6] > 0))  # nested masks


def test_batch_shapes_and_halves():
    s = synth.batch_shapes(64, 0)
    assert len(s) == 64 and set(s) <= set(synth.BATCH_SIZES)
    x = np.array([1.0, -2.5, 3.14159, 1e-3], dtype=np.float32)
    assert np.allclose(synth.bf16_to_f32(synth.to_bf16(x)), x, rtol=2 ** -8)
    assert np.allclose(synth.f16_to_f32(synth.to_f16(x)), x, rtol=2 ** -11)
