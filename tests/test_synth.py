"""The seeded input module: generators and storage-format conversions.

Both the CUDA path and the oracle receive their inputs from `synth`, so its conversions are
pinned here against independent references: torch's bfloat16 and float8_e4m3fn casts, which
round to nearest even, and the formats' definitions for saturation and NaN. Inputs are exact
in binary32, so torch's cast rounds once, as synth does. Also pinned: every code decodes as
torch decodes it and encodes back to itself; the uniform stream lies on [-1, 1) on the
2^-52 grid whatever the chunking; and the threaded normal generator equals the serial one
bit for bit.
"""
import numpy as np
import pytest

import synth as S

torch = pytest.importorskip("torch")


def _f32_exact_values(seed, n, lo_exp, hi_exp):
    """binary32 values (as binary64) over a wide exponent range, both signs, with exact
    ties for the 8- and 4-significant-bit formats mixed in."""
    rng = np.random.default_rng(seed)
    sig = rng.integers(1 << 23, 1 << 24, size=n).astype(np.float64)  # 24-bit significands
    exp = rng.integers(lo_exp, hi_exp, size=n)
    x = np.ldexp(sig, exp - 23) * np.where(rng.random(n) < 0.5, -1.0, 1.0)
    ties8 = np.ldexp(rng.integers(1 << 8, 1 << 9, size=n // 4) * 2.0 + 1.0, -9)   # (2k+1)/512 in [1, 2)
    ties4 = np.ldexp(rng.integers(1 << 4, 1 << 5, size=n // 4) * 2.0 + 1.0, -5)   # (2k+1)/32 in [1, 2)
    scale = np.ldexp(1.0, rng.integers(lo_exp // 2, hi_exp // 2, size=n // 4))
    out = np.concatenate([x, ties8 * scale, ties4 * scale, [0.0, -0.0]])
    with np.errstate(over="ignore"):
        return out.astype(np.float32).astype(np.float64)  # exact in binary32 (subnormals included)


def test_bf16_encoding_rounds_like_torch():
    x = _f32_exact_values(1, 40000, -140, 128)
    x = np.concatenate([x, [np.inf, -np.inf, 3.4e38, -3.4e38]])
    got = S.to_bf16_bits(x)
    ref = torch.from_numpy(x.astype(np.float32)).to(torch.bfloat16).view(torch.int16).numpy().astype(np.uint16)
    assert np.array_equal(got, ref)
    nan = S.to_bf16_bits(np.array([np.nan]))
    assert np.isnan(S.bf16_bits_to_f64(nan))[0]


def test_e4m3_encoding_rounds_like_torch_and_saturates():
    x = _f32_exact_values(2, 40000, -14, 9)
    x = x[np.abs(x) <= 448.0]
    got = S.to_e4m3_bits(x)
    ref = torch.from_numpy(x.astype(np.float32)).to(torch.float8_e4m3fn).view(torch.uint8).numpy()
    assert np.array_equal(got, ref)
    # beyond the largest finite value (448 = 0x7E) the encoding saturates; NaN is 0x7F
    assert list(S.to_e4m3_bits(np.array([500.0, 1e9, -1e9, np.inf]))) == [0x7E, 0x7E, 0xFE, 0x7E]
    assert S.to_e4m3_bits(np.array([np.nan]))[0] & 0x7F == 0x7F


@pytest.mark.filterwarnings("ignore:invalid value encountered in cast:RuntimeWarning")
def test_every_code_decodes_like_torch_and_encodes_back():
    codes8 = np.arange(256, dtype=np.uint8)
    dec8 = S.e4m3_bits_to_f64(codes8)
    ref8 = torch.from_numpy(codes8).view(torch.float8_e4m3fn).to(torch.float64).numpy()
    assert np.array_equal(np.isnan(dec8), np.isnan(ref8)) and np.array_equal(dec8[~np.isnan(dec8)],
                                                                                   ref8[~np.isnan(ref8)])
    fin8 = ~np.isnan(dec8)
    assert np.array_equal(S.to_e4m3_bits(dec8[fin8]), codes8[fin8])

    codes16 = np.arange(1 << 16, dtype=np.uint32).astype(np.uint16)
    dec16 = S.bf16_bits_to_f64(codes16)
    ref16 = torch.from_numpy(codes16.view(np.int16)).view(torch.bfloat16).to(torch.float64).numpy()
    assert np.array_equal(np.isnan(dec16), np.isnan(ref16))
    fin16 = ~np.isnan(dec16)
    assert np.array_equal(dec16[fin16], ref16[fin16])
    assert np.array_equal(S.to_bf16_bits(dec16[fin16]), codes16[fin16])


def test_uniform_stream_grid_range_and_chunking():
    a = S.uniform(7, 3, 100003)
    assert a.min() >= -1.0 and a.max() < 1.0
    assert np.array_equal(np.ldexp(a + 1.0, 52), np.rint(np.ldexp(a + 1.0, 52)))  # on the 2^-52 grid
    assert np.array_equal(a, S.uniform(7, 3, 100003, chunk=997))
    assert not np.array_equal(a, S.uniform(7, 4, 100003))  # another matrix id, another stream
    assert abs(a.mean()) < 0.01 and abs(a.var() - 1.0 / 3.0) < 0.01


def test_threaded_normal_equals_serial_bitwise():
    count = 2 * (1 << 22) + 2 * 1001 + 1  # three chunks of pairs, odd count
    z1 = S.normal(11, 0, count, threads=1)
    z4 = S.normal(11, 0, count, threads=4)
    assert np.array_equal(z1, z4)
    assert abs(z1.mean()) < 0.01 and abs(z1.std() - 1.0) < 0.01


def test_randint_and_pow2_scales_cover_their_stated_ranges():
    r = S.randint(5, 1, 200000, -4, 4)
    assert r.min() == -4 and r.max() == 4 and set(np.unique(r)) == set(range(-4, 5))
    counts = np.bincount(r + 4)
    assert counts.min() > 0.9 * counts.mean()  # roughly uniform
    p = S.pow2_row_scales(5, 2, 100000)
    m, e = np.frexp(p)
    assert np.all(m == 0.5)  # exact powers of two
    assert set(np.unique(e - 1)) == set(range(-8, 9))
