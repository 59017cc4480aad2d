"""CPU model of the word arithmetic of the 1-byte split and last-pair passes,
checked against the oracle.

At 1-byte symbols these passes replace per-symbol work by word arithmetic:

  pass A     bit k of four bytes gathered into a nibble by one multiply,
             ((q >> k) & 0x01010101) * 0x10204080 >> 28; each thread reads
             its 16-byte chunks starting at a lane-dependent chunk and the
             packed bits are rotated back with funnel shifts;
  pass B     a lane's 8 symbols stably partitioned in registers by two byte
             permutes whose selectors come from a 256-entry table indexed by
             the symbols' 8 bits; byte i is then stored at the zeros'
             pointer + i (i < nz) or at the ones' pointer + i - nz;
  last pair  the 8 next-level bits spread to one per byte (a multiply and a
             mask per 4 bits), reordered by the same byte permutes and
             gathered back (a multiply): the zeros' bits, then the ones'.

This model applies the same constants and selectors with numpy (the byte
permute and the funnel shift emulated from their definitions) and compares
the words, staged symbols and bit streams they give with the oracle's
bitmaps (Fig. 1: a level's bits, then the stable split by them), so a wrong
constant, selector or rotation fails here on the CPU.
"""
import numpy as np
import pytest

from oracle import serialwt
from paper_1407_8142_gb300 import synth

M32 = 0xFFFFFFFF


def byte_perm(x, y, s):
    """Byte permute (default mode): byte i of the result is byte
    (s >> 4i) & 7 of the 8-byte value y:x."""
    x, y, s = (np.asarray(a, dtype=np.uint64) for a in (x, y, s))
    src = [(x >> np.uint64(8 * j)) & np.uint64(0xFF) for j in range(4)] + \
          [(y >> np.uint64(8 * j)) & np.uint64(0xFF) for j in range(4)]
    src = np.stack(np.broadcast_arrays(*src))
    r = np.zeros(src.shape[1:], dtype=np.uint64)
    for i in range(4):
        nib = ((s >> np.uint64(4 * i)) & np.uint64(0xF)).astype(np.int64)
        assert np.all(nib < 8), "selectors name bytes 0..7 only"
        r |= np.take_along_axis(src, np.broadcast_to(nib, src.shape[1:])[None], 0)[0] << np.uint64(8 * i)
    return r.astype(np.uint64)


def funnelshift_l(lo: int, hi: int, sh: int) -> int:
    """Upper 32 bits of (hi:lo) shifted left by sh mod 32."""
    return ((((hi & M32) << 32) | (lo & M32)) << (sh & 31)) >> 32 & M32


def selectors() -> np.ndarray:
    """Table entry m: output byte o names the o-th byte of the stable
    partition of bytes 0..7 by the bits of m (clear first, then set)."""
    out = np.zeros(256, dtype=np.uint64)
    for m in range(256):
        order = [j for j in range(8) if not (m >> j) & 1] + [j for j in range(8) if (m >> j) & 1]
        out[m] = sum(j << (4 * o) for o, j in enumerate(order))
    return out


def gather4(q, k, magic=0x10204080):
    """Bit k of the four bytes of q as a nibble (bit j: byte j)."""
    q = np.asarray(q, dtype=np.uint64)
    x = (q >> np.uint64(k)) & np.uint64(0x01010101)
    return ((x * np.uint64(magic)) & np.uint64(M32)) >> np.uint64(28)


def thread_words(chunk_bytes: np.ndarray, lane: int, k: int, wpt: int, rot_bug: int = 0) -> list[int]:
    """The thread's wpt bit words from its 32*wpt consecutive bytes, read as
    2*wpt 16-byte chunks starting at chunk r and rotated back (rot_bug plants
    a rotation back by a different amount than the read's)."""
    nc = 2 * wpt
    r = (lane // (8 // nc)) & (nc - 1)
    words = chunk_bytes.view("<u4").astype(np.uint64)  # 4 words per chunk
    p = []
    for j in range(nc):
        c = (j + r) & (nc - 1)
        bits = 0
        for m in range(4):
            bits |= int(gather4(words[4 * c + m], k)) << (4 * m)
        p.append(bits)
    r = (r + rot_bug) & (nc - 1)
    if wpt == 1:
        v = p[0] | (p[1] << 16)
        return [funnelshift_l(v, v, 16 * r)]
    lo, hi = p[0] | (p[1] << 16), p[2] | (p[3] << 16)
    if r & 2:
        lo, hi = hi, lo
    sh = 16 * (r & 1)
    return [funnelshift_l(hi, lo, sh), funnelshift_l(lo, hi, sh)]


def level_words(S: np.ndarray, k: int) -> np.ndarray:
    """Bit k of every symbol, packed LSB-first into 32-bit words."""
    by = np.packbits(((S.astype(np.uint32) >> k) & 1).astype(np.uint8), bitorder="little")
    return by.view("<u4")


def pext8(v: int, m: int) -> int:
    """The bits of v where m is set, packed from bit 0 in order."""
    out, o = 0, 0
    for j in range(8):
        if (m >> j) & 1:
            out |= ((v >> j) & 1) << o
            o += 1
    return out


def last_pair_compact(m, v, spread=0x00204081, gather=0x10204080):
    """Level-(L-1) bits v of 8 symbols, reordered by their level-(L-2) bits
    m: the zeros' bits, then the ones' (bit j of the result)."""
    m = np.asarray(m, dtype=np.uint64)
    v = np.asarray(v, dtype=np.uint64)
    sel = selectors()[m.astype(np.int64)]
    slo = ((v & np.uint64(15)) * np.uint64(spread)) & np.uint64(0x01010101)
    shi = ((v >> np.uint64(4)) * np.uint64(spread)) & np.uint64(0x01010101)
    plo = byte_perm(slo, shi, sel & np.uint64(0xFFFF))
    phi = byte_perm(slo, shi, sel >> np.uint64(16))
    g = np.uint64(gather)
    return (((plo * g) & np.uint64(M32)) >> np.uint64(28)) | ((((phi * g) & np.uint64(M32)) >> np.uint64(28)) << np.uint64(4))


# ---------------------------------------------------------------- pass A

@pytest.mark.parametrize("k", range(8))
def test_nibble_gather_is_bit_k_of_each_byte(k):
    rng = np.random.default_rng(k)
    q = rng.integers(0, 1 << 32, 20000, dtype=np.uint64)
    want = sum((((q >> np.uint64(8 * j + k)) & np.uint64(1)) << np.uint64(j)) for j in range(4))
    assert np.array_equal(gather4(q, k), want)


@pytest.mark.parametrize("wpt", [1, 2])
@pytest.mark.parametrize("sigma,kind", [(256, "zipf"), (256, "uniform"), (7, "runs")])
def test_rotated_loads_give_the_oracle_words(wpt, sigma, kind):
    # a warp of 32 threads over 32*wpt bytes each: every thread's words must
    # be level 0's bitmap words at its position (every rotation 0..2wpt-1
    # occurs), and bit k of its bytes for every k
    n = 32 * 32 * wpt
    S = synth.pattern(kind, n, sigma, 1, seed=wpt).astype(np.uint8)
    ref = serialwt.build(S, sigma)
    L = serialwt.levels(sigma)
    for lane in range(32):  # level 0: bit L-1 of S itself
        chunk = S[32 * wpt * lane: 32 * wpt * (lane + 1)]
        got = thread_words(chunk, lane, L - 1, wpt)
        assert got == [int(w) for w in ref["bits"][0][wpt * lane: wpt * (lane + 1)]]
    for k in range(8):  # and bit k of the same bytes, for every k
        for lane in range(32):
            chunk = S[32 * wpt * lane: 32 * wpt * (lane + 1)]
            assert thread_words(chunk, lane, k, wpt) == [int(w) for w in level_words(chunk, k)]


# ---------------------------------------------------------------- pass B

def test_partition_selectors_split_every_pattern_stably():
    sel = selectors()
    rng = np.random.default_rng(1)
    x = rng.integers(0, 1 << 32, 256, dtype=np.uint64)
    y = rng.integers(0, 1 << 32, 256, dtype=np.uint64)
    lo = byte_perm(x, y, sel & np.uint64(0xFFFF))
    hi = byte_perm(x, y, sel >> np.uint64(16))
    for i in range(256):
        src = [(int(x[i]) >> (8 * j)) & 0xFF for j in range(4)] + [(int(y[i]) >> (8 * j)) & 0xFF for j in range(4)]
        want = [src[j] for j in range(8) if not (i >> j) & 1] + [src[j] for j in range(8) if (i >> j) & 1]
        got = [(int(lo[i]) >> (8 * j)) & 0xFF for j in range(4)] + [(int(hi[i]) >> (8 * j)) & 0xFF for j in range(4)]
        assert got == want


def pass_b_stage(seg: np.ndarray, k: int, wpt: int = 2) -> np.ndarray:
    """One warp's segment (1024*wpt symbols, 8 per lane per step) staged as
    the split pass does it: zeros from offset 0, ones after the zeros."""
    n = seg.size
    words = level_words(seg, k)
    pre = np.concatenate([[0], np.cumsum([bin(int(w)).count("1") for w in words])[:-1]])  # ones before each word
    nz_total = n - int(sum(bin(int(w)).count("1") for w in words))
    stage = np.full(n, -1, dtype=np.int64)
    sel = selectors()
    zbase, obase = 0, nz_total
    for s in range(32 * wpt // 8):
        for lane in range(32):
            pos0 = 256 * s + 8 * lane
            wsub = pos0 // 32
            wx, wy = int(words[wsub]), int(pre[wsub])
            bo = (lane % 4) * 8
            m = int(byte_perm(wx, 0, 0x4440 | (lane & 3)))  # the lane's 8 bits
            grp = seg[pos0:pos0 + 8].view("<u4").astype(np.uint64)
            lo = int(byte_perm(grp[0], grp[1], sel[m] & np.uint64(0xFFFF)))
            hi = int(byte_perm(grp[0], grp[1], sel[m] >> np.uint64(16)))
            nz = 8 - bin(m).count("1")
            Rl = wy + bin(wx & ((1 << bo) - 1)).count("1")  # ones before pos0 in the warp
            za = zbase + (pos0 - Rl)
            ob = obase + Rl - nz
            for i in range(8):
                v = ((lo if i < 4 else hi) >> (8 * (i & 3))) & 0xFF
                addr = (za if i < nz else ob) + i
                assert stage[addr] == -1, "two symbols staged at one place"
                stage[addr] = v
    return stage


@pytest.mark.parametrize("sigma,kind,seed", [(256, "zipf", 0), (256, "uniform", 1), (2, "uniform", 2),
                                             (256, "sorted", 3), (64, "runs", 4)])
def test_pass_b_stages_the_oracle_split(sigma, kind, seed):
    # one warp segment of 2048 symbols that is the whole sequence: level 0
    # has one node, so the staged zeros-then-ones are T_1, whose bit L-2
    # must be the oracle's B_1
    S = synth.pattern(kind, 2048, sigma, 1, seed=seed).astype(np.uint8)
    L = serialwt.levels(sigma)
    stage = pass_b_stage(S, L - 1)
    bit = (S.astype(np.int64) >> (L - 1)) & 1
    assert np.array_equal(stage, np.concatenate([S[bit == 0], S[bit == 1]]).astype(np.int64))
    if L >= 2:
        ref = serialwt.build(S, sigma)
        w1 = level_words(stage.astype(np.uint8), L - 2)
        assert np.array_equal(w1, ref["bits"][1][:w1.size])


# ---------------------------------------------------------------- last pair

def test_last_pair_compaction_every_pattern():
    m, v = np.meshgrid(np.arange(256), np.arange(256), indexing="ij")
    got = last_pair_compact(m.ravel(), v.ravel())
    want = np.array([pext8(int(b), 255 ^ int(a)) | (pext8(int(b), int(a)) << (8 - bin(int(a)).count("1")))
                     for a, b in zip(m.ravel(), v.ravel())], dtype=np.uint64)
    assert np.array_equal(got, want)


def last_pair_streams(S: np.ndarray, L: int):
    """The zeros' and ones' level-(L-1) bit streams of one warp-sized
    sequence, 8 symbols at a time, by the compaction above."""
    w0, w1 = level_words(S, 1), level_words(S, 0)  # bits of levels L-2 and L-1
    zs, os_ = [], []
    for a, b in zip(w0, w1):
        for byte in range(4):
            m, v = (int(a) >> (8 * byte)) & 0xFF, (int(b) >> (8 * byte)) & 0xFF
            P = int(last_pair_compact(m, v))
            c1 = bin(m).count("1")
            zs += [(P >> j) & 1 for j in range(8 - c1)]
            os_ += [(P >> j) & 1 for j in range(8 - c1, 8)]
    return zs, os_


@pytest.mark.parametrize("top,kind,seed", [(0, "uniform", 0), (5, "zipf", 1), (63, "runs", 2)])
def test_last_pair_streams_are_the_oracles_last_level(top, kind, seed):
    # symbols 4*top + (0..3) of an 8-level alphabet: levels 0..5 have one
    # node each, so level 7 of the oracle is the level-7 bits of the level-6
    # zeros, in order, then those of its ones
    n = 2048
    S = (4 * top + synth.pattern(kind, n, 4, 1, seed=seed).astype(np.int64)).astype(np.uint8)
    ref = serialwt.build(S, 256)
    zs, os_ = last_pair_streams(S, 8)
    row = np.array(zs + os_, dtype=np.uint8)
    by = np.packbits(row, bitorder="little").view("<u4")
    assert np.array_equal(by, ref["bits"][7][:by.size])


def test_model_catches_planted_mistakes():
    # each planted mistake must make the model disagree with the oracle's
    # bits or with the definition
    S = synth.pattern("zipf", 2048, 4, 1, seed=7).astype(np.uint8)
    m, v = np.meshgrid(np.arange(256), np.arange(256), indexing="ij")
    good = last_pair_compact(m.ravel(), v.ravel())
    assert not np.array_equal(last_pair_compact(m.ravel(), v.ravel(), spread=0x00204080), good)
    assert not np.array_equal(last_pair_compact(m.ravel(), v.ravel(), gather=0x10204000), good)
    q = np.random.default_rng(3).integers(0, 1 << 32, 1000, dtype=np.uint64)
    assert not np.array_equal(gather4(q, 3, magic=0x08102040), gather4(q, 3))
    chunk = S[64:128]
    assert any(thread_words(chunk, lane, 0, 2, rot_bug=1) != [int(w) for w in level_words(chunk, 0)]
               for lane in range(32))
