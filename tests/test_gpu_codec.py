"""The value codecs of the 16-bit storage formats (lbps_codec16), which run
the same conversion routines the time step stores and loads the pair sums
with, checked against each format's definition written out here: IEEE half
through numpy's float16, bfloat16 as the upper half of an FP32 word rounded
to nearest even, BFP13 from its definition (two values in a 32-bit word
sharing a 4-bit exponent E, each a sign and a 13-bit magnitude m, value
m 2^(E-13); E the smallest exponent at which both magnitudes round to at most
8191; E = 15 with m = 8191: infinity).  Stochastic rounding of the IEEE-type
formats: each result one of the two neighbours, unbiased on average,
deterministic in the value and the key."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

HALVES = ("bf16", "f16")


@pytest.fixture(scope="module")
def L():
    assert torch.cuda.is_available(), "GPU tests need a CUDA device"
    from paper_2301_00228_gb300 import lbps
    return lbps


def half_value(fmt, code):
    code = np.asarray(code, np.uint32)
    with np.errstate(invalid="ignore"):
        if fmt == "f16":
            return code.astype(np.uint16).view(np.float16).astype(np.float64)
        return (code << 16).view(np.float32).astype(np.float64)


def half_nearest(fmt, x):
    """Round-to-nearest-even code of FP32 values x."""
    x = np.asarray(x, np.float32)
    if fmt == "f16":
        with np.errstate(over="ignore"):
            return x.astype(np.float16).view(np.uint16).astype(np.uint32)
    u = x.view(np.uint32).astype(np.uint64)
    return (((u + 0x7FFF + ((u >> 16) & 1)) >> 16) & 0xFFFF).astype(np.uint32)


def bfp13_values(w):
    """(Nx, Ny) of 32-bit BFP13 words, by the definition."""
    w = np.asarray(w, np.int64)
    e = w >> 28
    ma, mb = (w >> 14) & 0x1FFF, w & 0x1FFF
    out = []
    for m, sbit in ((ma, 27), (mb, 13)):
        v = np.ldexp(m.astype(np.float64), (e - 13).astype(np.int32))
        v = np.where((e == 15) & (m == 8191), np.inf, v)
        out.append(np.where((w >> sbit) & 1, -v, v))
    return out


def bfp13_nearest(a, b):
    """BFP13 words of FP32 value pairs by the definition: the first E at which
    both rounded magnitudes fit in 13 bits; both infinite if either value is
    not below 32762 (which rounds onto the infinity pattern or beyond)."""
    a, b = np.asarray(a, np.float32), np.asarray(b, np.float32)
    xa, xb = np.abs(a.astype(np.float64)), np.abs(b.astype(np.float64))
    signs = (np.signbit(a).astype(np.int64) << 27) | (np.signbit(b).astype(np.int64) << 13)
    word = np.full(a.shape, -1, np.int64)
    for e in range(16):
        ma, mb = np.rint(xa * 2.0 ** (13 - e)), np.rint(xb * 2.0 ** (13 - e))
        take = (word < 0) & (np.maximum(ma, mb) <= 8191) & (xa < 32762) & (xb < 32762)
        word = np.where(take, (e << 28) | (np.nan_to_num(ma).astype(np.int64) << 14) |
                        np.nan_to_num(mb).astype(np.int64), word)
    word = np.where(word < 0, 0xF7FFDFFF, word)
    return (word | signs).astype(np.uint32)


def encode(L, fmt, x, key0=0, sr=False):
    xs = torch.from_numpy(np.asarray(x, np.float32).copy()).cuda()
    c = torch.empty(xs.numel(), dtype=torch.int16, device="cuda")
    L.lbps_codec16(fmt, 1, xs.data_ptr(), c.data_ptr(), xs.numel(), key0, sr)
    torch.cuda.synchronize()
    return c.cpu().numpy().view(np.uint16).astype(np.uint32)


def decode(L, fmt, codes):
    c = torch.from_numpy(np.asarray(codes, np.uint16).view(np.int16).copy()).cuda()
    out = torch.empty(c.numel(), dtype=torch.float32, device="cuda")
    L.lbps_codec16(fmt, 0, out.data_ptr(), c.data_ptr(), c.numel())
    torch.cuda.synchronize()
    return out.cpu().numpy()


def bfp13_encode(L, a, b):
    x = np.stack([np.asarray(a, np.float32), np.asarray(b, np.float32)], -1).ravel()
    codes = encode(L, "bfp13", x)
    return (codes[0::2] | (codes[1::2] << 16)).astype(np.uint32)


def bfp13_decode(L, words):
    words = np.asarray(words, np.uint32)
    codes = np.stack([words & 0xFFFF, words >> 16], -1).ravel()
    x = decode(L, "bfp13", codes).astype(np.float64)
    return x[0::2], x[1::2]


def samples(seed=0):
    rng = np.random.default_rng(seed)
    x = np.concatenate([rng.uniform(-1, 1, 200_000), rng.standard_normal(200_000) * 2.0 ** 10,
                        np.exp(rng.uniform(-30, 12, 200_000)) * rng.choice([-1, 1], 200_000),
                        rng.uniform(32_000, 33_000, 20_000), rng.uniform(65_000, 66_000, 20_000),
                        [0.0, -0.0, 1.0, -1.0, 0.5, 2.0 ** -13, 3 * 2.0 ** -14, 32_752, 32_756, 32_760, 32_762,
                         65_504, 65_520, 1e30, -1e30, np.inf, -np.inf]])
    return x.astype(np.float32)


@pytest.mark.parametrize("fmt", HALVES)
def test_decode_every_code(L, fmt):
    codes = np.arange(65536, dtype=np.uint32)
    got = decode(L, fmt, codes).astype(np.float64)
    want = half_value(fmt, codes)
    nan = np.isnan(want)
    assert np.array_equal(np.isnan(got), nan)
    assert np.array_equal(got[~nan], want[~nan])
    assert np.array_equal(np.signbit(got[~nan]), np.signbit(want[~nan]))


@pytest.mark.parametrize("fmt", HALVES)
def test_encode_round_trip(L, fmt):
    codes = np.arange(65536, dtype=np.uint32)
    vals = half_value(fmt, codes)
    keep = np.isfinite(vals)
    assert np.array_equal(encode(L, fmt, vals[keep]), codes[keep])


@pytest.mark.parametrize("fmt", HALVES)
def test_encode_nearest(L, fmt):
    x = samples()
    # the midpoints between neighbouring finite values (ties to even)
    v = half_value(fmt, np.arange(0x7FFF))
    v = np.unique(v[np.isfinite(v)])
    mid = (v[:-1] + v[1:]) / 2
    x = np.concatenate([x, mid[mid.astype(np.float32).astype(np.float64) == mid].astype(np.float32)])
    assert np.array_equal(encode(L, fmt, x), half_nearest(fmt, x))


@pytest.mark.parametrize("fmt", HALVES)
def test_stochastic_rounding(L, fmt):
    """Every result is one of the two neighbours of the value; over many keys
    the share rounded up is the value's fraction of the step; the same value
    and key give the same code."""
    rng = np.random.default_rng(5)
    n = 1 << 16
    lo_code = {"f16": 0x5000 + 333, "bf16": 0x4480 + 17}[fmt]   # finite, mid-range
    lo, hi = half_value(fmt, np.array([lo_code, lo_code + 1]))
    for frac in (0.1, 0.5, 0.73):
        val = np.float32(lo + frac * (hi - lo))
        codes = encode(L, fmt, np.full(n, val, np.float32), key0=int(rng.integers(0, 1 << 30)), sr=True)
        assert set(np.unique(codes)) <= {lo_code, lo_code + 1}
        p_up = (codes == lo_code + 1).mean()
        want = (float(val) - lo) / (hi - lo)
        assert abs(p_up - want) <= 5 * np.sqrt(want * (1 - want) / n) + 2.0 ** -12, (fmt, frac, p_up, want)
    x = samples(1)
    assert np.array_equal(encode(L, fmt, x, key0=12, sr=True), encode(L, fmt, x, key0=12, sr=True))


def bfp13_words(seed=0, n=1_000_000):
    rng = np.random.default_rng(seed)
    w = rng.integers(0, 1 << 32, n, dtype=np.uint64).astype(np.uint32)
    edge = [0, 0xF7FFDFFF, 0xFFFFFFFF, 0x0FFFFFFF, 0x1FFFFFFF, 0xF7FFC000, 0xF0001FFF, 0x80000000, 0x00002000]
    return np.concatenate([w, np.array(edge, np.uint32)])


def test_bfp13_decode(L):
    w = bfp13_words()
    a, b = bfp13_decode(L, w)
    ra, rb = bfp13_values(w)
    for got, want in ((a, ra), (b, rb)):
        assert np.array_equal(got, want)
        assert np.array_equal(np.signbit(got), np.signbit(want))


def test_bfp13_round_trip(L):
    """Every canonical word (E = 0, or the larger magnitude at least 4096,
    no infinity) comes back from its values unchanged."""
    w = bfp13_words(1)
    e, ma, mb = w >> 28, (w >> 14) & 0x1FFF, w & 0x1FFF
    inf = (e == 15) & ((ma == 8191) | (mb == 8191))
    w = w[~inf & ((e == 0) | (np.maximum(ma, mb) >= 4096))]
    a, b = bfp13_values(w)
    assert np.array_equal(bfp13_encode(L, a, b), w)


def test_bfp13_encode_nearest(L):
    rng = np.random.default_rng(3)
    n = 400_000
    a = samples(2)[:n]
    scale = 10.0 ** rng.uniform(-6, 0, a.size)                 # the partner smaller by up to 10^6
    b = (a * scale * rng.choice([-1, 1], a.size)).astype(np.float32)
    # values where the larger magnitude is at a rounding boundary of its
    # binade (the exponent steps up) and half-way cases
    e = rng.integers(0, 16, 5000)
    m = rng.integers(0, 8192, 5000)
    tie = (np.ldexp(m + 0.5, e - 13)).astype(np.float32)
    top = (np.ldexp(np.full(5000, 8191.5), e - 13) * (1 + rng.choice([-1e-7, 0, 1e-7], 5000))).astype(np.float32)
    a = np.concatenate([a, b, tie, top, [np.nan, 1.0, -np.inf, 32761.99, 32762.0]]).astype(np.float32)
    b = np.concatenate([b, a[:b.size], top[::-1], tie[::-1], [1.0, np.nan, 2.0, -1.0, 0.0]]).astype(np.float32)
    got = bfp13_encode(L, a, b)
    assert np.array_equal(got, bfp13_nearest(a, b))
    # NaN and overflow give infinities in both slots, with the signs kept;
    # beside the largest finite magnitude a small value flushes to a signed 0
    x, y = bfp13_decode(L, got[-5:])
    assert np.all(np.isinf(x[[0, 1, 2, 4]])) and np.all(np.isinf(y[[0, 1, 2, 4]]))
    assert np.signbit(x[2]) and not np.signbit(y[2])
    assert x[3] == 32760.0 and y[3] == 0.0 and np.signbit(y[3])


def test_codec_arguments(L):
    x = torch.zeros(4, device="cuda")
    c = torch.zeros(4, dtype=torch.int16, device="cuda")
    for args in (("f32", 1, x.data_ptr(), c.data_ptr(), 4), ("f16", 2, x.data_ptr(), c.data_ptr(), 4),
                 ("f16", 1, 0, c.data_ptr(), 4), ("f16", 1, x.data_ptr(), c.data_ptr(), -1),
                 ("bfp13", 1, x.data_ptr(), c.data_ptr(), 3), ("bfp13", 1, x.data_ptr() + 4, c.data_ptr(), 2)):
        with pytest.raises(L.LbpsError) as e:
            L.lbps_codec16(*args)
        assert e.value.code == L.LBPS_ERR_INVALID
    L.lbps_codec16("bfp13", 1, 0, 0, 0)   # nothing to do
