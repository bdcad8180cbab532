"""The seeded input generators: the counter-based splitmix64 against the
published SplitMix64 sequence, determinism and stream separation, and the value
distributions each workload's input is stated to have."""

import numpy as np

from paper_2012_07145_gb300 import synth

GOLDEN = 0x9E3779B97F4A7C15


def test_splitmix64_reproduces_the_published_sequence():
    # SplitMix64 seeded with 0 outputs mix(k * golden) for k = 1, 2, 3; the
    # counter form mixes (n + golden), so counters 0, golden, 2 golden give them
    ctr = np.array([0, GOLDEN, (2 * GOLDEN) % 2 ** 64], dtype=np.uint64)
    with np.errstate(over="ignore"):
        out = synth.splitmix64(ctr)
    assert [int(v) for v in out] == [0xE220A8397B1DCDAF, 0x6E789E6AA1B965F4, 0x06C45D188009454F]


def test_determinism_and_stream_separation():
    a = synth.uniform_f32((3, 17, 29), seed=5, stream=2)
    assert np.array_equal(a, synth.uniform_f32((3, 17, 29), seed=5, stream=2))
    assert not np.array_equal(a, synth.uniform_f32((3, 17, 29), seed=6, stream=2))
    assert not np.array_equal(a, synth.uniform_f32((3, 17, 29), seed=5, stream=3))
    # element n depends only on (seed, stream, n): a prefix of a larger draw
    big = synth.uniform_f32((1000,), seed=5, stream=2)
    assert np.array_equal(synth.uniform_f32((400,), seed=5, stream=2), big[:400])


def test_uniform_values_are_exact_24_bit_fractions_in_unit_interval():
    u = synth.uniform_f32((1 << 18,), seed=1)
    assert u.dtype == np.float32 and u.min() >= 0.0 and u.max() < 1.0
    assert np.array_equal(u * np.float32(2 ** 24), np.floor(u * np.float32(2 ** 24)))
    assert abs(float(u.mean()) - 0.5) < 0.005 and abs(float(u.var()) - 1.0 / 12.0) < 0.002


def test_gaussian_moments():
    g = synth.gaussian_f64((1 << 18,), seed=2, stream=3)
    assert abs(g.mean()) < 0.01 and abs(g.std() - 1.0) < 0.01
    assert abs(np.mean(np.abs(g) < 1.0) - 0.6827) < 0.005


def test_workload_inputs_have_their_stated_distributions():
    h, w = 256, 384
    u8 = synth.gray_u8_lowcontrast(h, w)
    assert u8.dtype == np.uint8 and u8.shape == (1, h, w)
    assert abs(u8.mean() - 100.0) < 0.5 and abs(u8.std() - 20.0) < 0.5
    ll = synth.rgb_u16_gradient_noise(h, w)
    assert ll.dtype == np.uint16 and ll.shape == (3, h, w)
    r = ll[0].astype(np.float64) / 65535.0
    ramp = np.arange(w) / (w - 1)
    assert np.abs(r.mean(axis=0) - ramp)[8:-8].max() < 0.01      # R follows x/(W-1) (noise sigma 0.02)
    rgba = synth.rgba_sparse_f32(h, w)
    assert rgba.shape == (4, h, w) and set(np.unique(rgba[3]).tolist()) == {0.0, 1.0}
    assert abs(rgba[3].mean() - 0.25) < 0.01
    bg = synth.gray_f32_gradient_noise(h, w)
    assert bg.dtype == np.float32 and bg.min() >= 0.0 and bg.max() <= 1.0
    base = (np.arange(w)[None, :] / (w - 1) + np.arange(h)[:, None] / (h - 1)) / 2.0
    inner = (base > 0.2) & (base < 0.8)                           # away from the clamps
    assert abs(float((bg[0] - base)[inner].std()) - 0.05) < 0.002
