"""Pins of the oracle's stored-precision emulation against PyTorch's own
BF16 and FP8-E4M3 conversions (both round to nearest, ties to even)."""
import numpy as np
import torch

from oracle import storage


def _values(n=200_000, seed=0):
    rng = np.random.default_rng(seed)
    x = rng.standard_normal(n).astype(np.float32) * np.float32(10.0) ** rng.integers(-8, 8, n)
    edge = np.array([0.0, -0.0, 1.0, 1.00390625, 1.01171875, 3.140625, 65504.0, 1e-30, -2.5],
                    dtype=np.float32)
    return np.concatenate([x.astype(np.float32), edge])


def test_bf16_rounding_matches_torch():
    x = _values()
    ours = storage.bf16_round(x)
    ref = torch.from_numpy(x).to(torch.bfloat16).to(torch.float32).numpy()
    assert np.array_equal(ours.view(np.uint32), ref.view(np.uint32))


def test_e4m3_rounding_matches_torch_within_range():
    rng = np.random.default_rng(1)
    y = np.clip(rng.standard_normal(200_000) * 60, -448, 448).astype(np.float32)
    y = np.concatenate([y, np.float32([0, 2.0 ** -9, 2.0 ** -10, 3 * 2.0 ** -10, 448, -448,
                                       0.015625, 0.0146484375, 240, 232, 248])])
    ours = storage.e4m3_round(y)
    ref = torch.from_numpy(y).to(torch.float8_e4m3fn).to(torch.float64).numpy()
    assert np.array_equal(ours, ref)


def test_e4m3_saturates():
    assert storage.e4m3_round(np.float32([500.0, -1e6]))[0] == 448.0
    assert storage.e4m3_round(np.float32([500.0, -1e6]))[1] == -448.0


def test_fp8_scale_maps_column_amax_to_448():
    rng = np.random.default_rng(2)
    x = (rng.standard_normal((1000, 8)) * np.arange(1, 9)).astype(np.float32)
    s = storage.fp8_scales(x)
    codes = storage.e4m3_round((x / s).astype(np.float32))
    assert np.all(np.abs(codes).max(0) == 448.0)
    st = storage.stored(x.astype(np.float64), "fp8")
    # relative error of an E4M3 normal value is at most 2^-4
    big = np.abs(x) > s * 2.0 ** -6
    assert np.all(np.abs(st[big] - x[big]) <= 2.0 ** -4 * np.abs(x[big]) * (1 + 1e-6))


def test_f32_and_f64_storage():
    x = np.array([[1.0 / 3.0, 2.0 ** 0.5]])
    assert np.array_equal(storage.stored(x, "f64"), x)
    assert np.array_equal(storage.stored(x, "f32"), x.astype(np.float32).astype(np.float64))
