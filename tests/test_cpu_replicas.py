"""CPU replicas of the GPU path's index arithmetic and number primitives (no GPU needed).

The s = 1/2 block kernels never decode or encode a row with the walk of Sec. 3.1 / 3.2:
they split a state's bit word into a high part h (sites K..N-1) and a low part l (sites
0..K-1) and use that the rank of Sec. 3.2 is additive over positions,
    index(h, l) = off(h) + rank_K(l),
with rank_K read from byte-chunk tables, rank_K(l) = U[popc(l)][l >> 8] + R0[l & 255], and
off(h) summed over the ones of h.  Each exchange target is formed from these pieces in one of
five ways (both ends in the low byte, both in the second low byte, across the two, across the
split, both high) and, in the spin-flip basis, through the complement block.  The replicas
below restate those formulas and check every target against the oracle's encode of the
exchanged state, for all states of small sectors and samples of the N = 32 sector, together
with the bounds of the shared-memory rows the low targets index.

The double-float and fixed-point primitives (csrc/ef64.cuh, host-compilable) are checked
against long double and exact integer arithmetic by tests/native/ef64_check.cc.
"""
import math
import os
import shutil
import subprocess

import numpy as np
import pytest

import oracle

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
CSRC = os.path.join(ROOT, "paper_0706_3293_gb300", "csrc")
BLK_XPAD = 128          # pad rows after a staged block (the zero row the kernels read for a failed exchange)


def test_ef64_primitives_against_long_double(tmp_path):
    gxx = shutil.which("g++")
    if gxx is None:
        pytest.skip("no g++")
    exe = str(tmp_path / "ef64_check")
    subprocess.check_call([gxx, "-O2", "-std=c++17", "-ffp-contract=off", "-I", CSRC, "-o", exe,
                           os.path.join(ROOT, "tests", "native", "ef64_check.cc")])
    r = subprocess.run([exe], capture_output=True, text=True, timeout=600)
    assert r.returncode == 0, r.stdout + r.stderr
    assert "violations" in r.stdout


# ---- the block decomposition ------------------------------------------------------------

def popc(x):
    return bin(x).count("1")


def byte_tables(K):
    """R0[b] = sum over the ones of byte b (ascending positions t, j = 1, 2, ..) of C(t, j);
    U[k][b1] = the same sum for the ones of the second part b1 = l >> 8 at positions 8 + t,
    counted after the k - popc(b1) ones of the low byte."""
    R0 = [0] * 256
    for b in range(256):
        j, s = 0, 0
        for t in range(8):
            if b >> t & 1:
                j += 1
                s += math.comb(t, j)
        R0[b] = s
    nb1 = 1 << (K - 8)
    U = [[0] * nb1 for _ in range(K + 1)]
    for k in range(K + 1):
        for b1 in range(nb1):
            j, s = k - popc(b1), 0
            if j < 0 or j > 8:
                continue
            for t in range(K - 8):
                if b1 >> t & 1:
                    j += 1
                    s += math.comb(8 + t, j)
            U[k][b1] = s
    return U, R0


def rank_low(U, R0, l, k):
    return U[k][l >> 8] + R0[l & 255]


def off(K, h, k):
    """Rank contribution of the high ones (Sec. 3.2): the ones of h at sites K + t, numbered on
    from the k ones of the low part."""
    o, cnt, t = 0, k, 0
    while h >> t:
        if h >> t & 1:
            cnt += 1
            o += math.comb(K + t, cnt)
        t += 1
    return o


def word_of(digits):
    return sum(int(a) << u for u, a in enumerate(digits))


def digits_of(w, N):
    return [(w >> u) & 1 for u in range(N)]


@pytest.mark.parametrize("K", [8, 10, 12, 15])
def test_byte_tables_are_the_colex_rank(K):
    """rank_K(l) from the two table reads equals the rank of l among the K-bit words of its
    popcount in increasing order (the order of Sec. 3 on the low sites)."""
    U, R0 = byte_tables(K)
    seen = [0] * (K + 1)
    for l in range(1 << K):
        k = popc(l)
        assert rank_low(U, R0, l, k) == seen[k], (K, l)
        seen[k] += 1


def ring_bonds(N, extra=()):
    b = [(u, (u + 1) % N) for u in range(N)] + [(u, (u + 2) % N) for u in range(N)] + list(extra)
    return [(min(p, q), max(p, q)) for p, q in b]


def kernel_target(N, K, U, R0, w, p, q):
    """Row index the block kernels gather from for the exchange of bond (p < q) at state w
    (bits of p and q differ), by the kernels' own formulas."""
    mask = (1 << K) - 1
    h, l = w >> K, w & mask
    k = popc(l)
    if q < K:                                    # low bond: a row of the same staged block
        pat = (1 << p) | (1 << q)
        l2 = l ^ pat
        if q < 8:                                # both ends in the low byte
            t = U[k][l >> 8] + R0[l2 & 255]
        elif p >= 8:                             # both in the second part
            t = R0[l & 255] + U[k][l2 >> 8]
        else:                                    # across the two
            t = U[k][l2 >> 8] + R0[l2 & 255]
        n = math.comb(K, k)
        assert 0 <= t < n, "a low target leaves its staged block"
        return off(K, h, k) + t
    if p < K:                                    # across the split: one bit on each side
        hq = q - K
        k2 = k + (1 if h >> hq & 1 else -1)
        assert 0 <= k2 <= K
        return off(K, h ^ (1 << hq), k2) + rank_low(U, R0, l ^ (1 << p), k2)
    h2 = h ^ ((1 << (p - K)) | (1 << (q - K)))   # both high: the same row of another block
    return off(K, h2, k) + rank_low(U, R0, l, k)


def flip_target(N, K, U, R0, w, p, q):
    """Spin-flip basis (M = 0): an exchange that moves site N-1 up leaves the representatives;
    the kernels gather row n - 1 - r of the complement block (index(flip w) = D - 1 -
    index(w)), i.e. base - r with base = off(~h2, K - k2) + C(K, k2) - 1."""
    mask = (1 << K) - 1
    H = N - K
    h, l = w >> K, w & mask
    k = popc(l)
    if p >= K:                                   # both high
        h2 = h ^ ((1 << (p - K)) | (1 << (q - K)))
        k2, l2 = k, l
    else:                                        # across the split (q = N - 1)
        h2 = h ^ (1 << (q - K))
        l2 = l ^ (1 << p)
        k2 = popc(l2)
    base = off(K, ~h2 & ((1 << H) - 1), K - k2) + math.comb(K, k2) - 1
    return base - rank_low(U, R0, l2, k2)


def check_sector(N, A, bonds, sample=None, seed=0):
    K = min(15, N - 2)
    U, R0 = byte_tables(K)
    ob = oracle.Basis(N, 1, A)
    idx = range(ob.dim) if sample is None else np.random.default_rng(seed).integers(0, ob.dim, sample)
    ntarget = 0
    for i in idx:
        i = int(i)
        d = ob.decode(i)
        w = word_of(d)
        h, l = w >> K, w & ((1 << K) - 1)
        assert off(K, h, popc(l)) + rank_low(U, R0, l, popc(l)) == i          # the row's own index
        for p, q in bonds:
            if (w >> p & 1) == (w >> q & 1):
                continue
            w2 = w ^ (1 << p) ^ (1 << q)
            want = ob.encode(digits_of(w2, N))
            assert kernel_target(N, K, U, R0, w, p, q) == want, (N, A, i, p, q)
            ntarget += 1
    assert ntarget > 0


@pytest.mark.parametrize("N", [10, 12, 14, 16])
def test_block_targets_all_states(orc, N):
    """Every row of several sectors, every bond of a J1-J2 ring plus long-range bonds (which
    reach every slot kind): the kernels' target index equals the oracle's encode."""
    bonds = ring_bonds(N, extra=[(0, N // 2), (1, N - 1), (3, N - 3), (2, 9)])
    for A in sorted({1, N // 2 - 1, N // 2, N - 2}):
        check_sector(N, A, bonds)


@pytest.mark.parametrize("N,A", [(24, 12), (28, 13), (32, 16), (32, 11)])
def test_block_targets_sampled_large(orc, N, A):
    """Sampled rows of large sectors (the N = 32 one is the bench workload), K = 15 split."""
    check_sector(N, A, ring_bonds(N, extra=[(0, 17), (5, N - 1), (14, 15)]), sample=600, seed=N + A)


@pytest.mark.parametrize("N", [10, 12, 14])
def test_flip_block_targets(orc, N):
    """Spin-flip basis: exchanges that carry site N-1 up from a representative land in the
    complement block at base - r, which is the row of the flipped state."""
    K = min(15, N - 2)
    U, R0 = byte_tables(K)
    ob = oracle.Basis(N, 1, N // 2)
    full = (1 << N) - 1
    bonds = [b for b in ring_bonds(N) if b[1] == N - 1]
    nchk = 0
    for i in range(ob.dim // 2):                 # representatives: site N-1 up (bit 0)
        w = word_of(ob.decode(i))
        assert not (w >> (N - 1)) & 1
        for p, q in bonds:
            if (w >> p & 1) == (w >> q & 1):
                continue
            w2 = w ^ (1 << p) ^ (1 << q)         # site N-1 now down: not a representative
            want = ob.encode(digits_of(~w2 & full, N))
            assert want == ob.dim - 1 - ob.encode(digits_of(w2, N))
            assert flip_target(N, K, U, R0, w, p, q) == want, (N, i, p, q)
            nchk += 1
    assert nchk > 0


def test_shared_rows_in_bounds():
    """The staged block holds max_block + BLK_XPAD rows; a low target indexes below C(K, k)
    <= max_block (checked in kernel_target) and a failed exchange reads the zero row
    max_block + BLK_XPAD - 1, inside the allocation, for every split K the plans use."""
    for K in range(8, 16):
        max_block = max(math.comb(K, k) for k in range(K + 1))
        assert max_block + BLK_XPAD - 1 < max_block + BLK_XPAD
        assert max_block <= 6435


# ---- triangles of low bonds in the target tables --------------------------------------------

def ring_triangles(K):
    """Edge-disjoint triangles of the J1-J2 low bonds, as the table builder takes them:
    sites (p, p+1, p+2) for even p, e1 = (p, p+1), e2 = (p+1, p+2) of class J1 sharing site
    p+1, e3 = (p, p+2) of class J2."""
    return [((p, p + 1), (p + 1, p + 2), (p, p + 2)) for p in range(0, K - 2, 2)]


@pytest.mark.parametrize("K", [10, 13, 15])
def test_triangle_encoding_of_low_exchanges(K):
    """For three sites joined by three bonds either no spin pair or exactly two differ, so
    the table stores two targets: the first allowed edge in the order e1, e2, e3 and the
    second.  The first is always an e1 or e2 exchange (class J1); the second is e2 (class J1)
    when the spins of the ends of e3 are parallel, else e3 (class J2), which the kernel reads
    off the row's own word.  Per class, the stored targets summed as the kernel sums them
    equal the allowed exchanges' targets, for every K-bit word."""
    tris = ring_triangles(K)
    rank = {}
    seen = [0] * (K + 1)
    for l in range(1 << K):
        rank[l] = seen[popc(l)]
        seen[popc(l)] += 1
    Z = -1                                           # the zero row: contributes nothing
    for l in range(1 << K):
        for e1, e2, e3 in tris:
            ok = [((l >> a) ^ (l >> b)) & 1 for a, b in (e1, e2, e3)]
            assert sum(ok) in (0, 2)
            tg = [rank[l ^ (1 << a) ^ (1 << b)] for a, b in (e1, e2, e3)]
            allowed = [t for t, v in zip(tg, ok) if v]
            o1, o2 = (allowed[0], allowed[1]) if allowed else (Z, Z)
            second_is_e3 = ((l >> e3[0]) ^ (l >> e3[1])) & 1
            cls_a = [x for x in (o1, o2 if not second_is_e3 else Z) if x != Z]
            cls_b = [o2] if second_is_e3 else []
            assert sorted(cls_a) == sorted(t for t, v in zip(tg[:2], ok[:2]) if v)
            assert sorted(cls_b) == sorted(t for t, v in zip(tg[2:], ok[2:]) if v)


# ---- the row value's rounding through the conversion unit ------------------------------------

def test_exponent_shift_rounding_matches_exact():
    """The block rows round s 2^k (s the exact int64 row sum, k the fixed-point unit) as
    round-to-nearest-even binary64 of s with its exponent field moved by k, whenever the
    result is a normal number.  Replica: Python's int -> float conversion (correctly
    rounded) with the field moved by k, against the exact rational s 2^k rounded by
    Fraction -> float, for random s over the whole int64 range and k over the range the
    kernels use; plus the cases at the ends of that range, which must fall back."""
    import struct
    from fractions import Fraction

    def bits(x):
        return struct.unpack("<Q", struct.pack("<d", x))[0]

    def shifted(s, k):
        """the kernel's fast path, or None where it hands over to the integer rounding"""
        if s == 0:
            return None
        b = bits(float(s))
        e = ((b >> 52) & 0x7FF) + k
        if not 1 <= e <= 2046:
            return None
        return (b + (k << 52)) & 0xFFFFFFFFFFFFFFFF

    rng = np.random.default_rng(5)
    n_fast = 0
    for _ in range(20000):
        nb = int(rng.integers(1, 64))
        s = int(rng.integers(0, 1 << 62)) >> (62 - nb) if nb < 62 else int(rng.integers(0, 1 << 62))
        s = -s if rng.integers(0, 2) else s
        # the kernels' k is the unit exponent E - 1075 (E about 1000..1023) plus that of g0;
        # a wide range besides, down to where the results leave the normal numbers
        k = int(rng.integers(-90, -40)) if rng.integers(0, 2) else int(rng.integers(-1140, 900))
        got = shifted(s, k)
        if got is None:
            continue
        n_fast += 1
        assert got == bits(float(Fraction(s) * Fraction(2) ** k)), (s, k)
    assert n_fast > 12000
    # ties: s with exactly 54 significant bits ending in ...1 (halfway), both parities
    for s in ((1 << 53) + 1, (1 << 53) + 3, -((1 << 60) + (1 << 7)), (1 << 62) + (1 << 8) + (1 << 9)):
        assert shifted(s, -1075) == bits(float(Fraction(s) * Fraction(2) ** -1075))
    # out of the normal range: the kernel hands over to the integer rounding
    assert shifted(1, -1075) is None and shifted(0, -1000) is None and shifted(1 << 62, 1000) is None
