// blk_sweep.cuh -- thread-per-row kernels of the s = 1/2 block path (layout in blk.cuh):
// the sweep over the blocks of a sector and the bodies of the matvec and Lanczos
// products.  Compiles under nvcc (blk.cu, generic row policy) and under NVRTC (jit.cu,
// bond slots written out per plan).
#pragma once

#include "blk_params.cuh"
#include "ef64.cuh"
#include "hm_dev.cuh"

namespace hm {

constexpr int BLK_NT = 512;

__host__ __device__ __forceinline__ size_t al16(size_t x) { return (x + 15) & ~(size_t)15; }

// ---------------------------------------------------------------------------------------
// Thread-per-row sweep over the blocks (matvec API and the Lanczos products)
//
// One thread per row of a block.  Every bond is a slot whose constants sit in the kernel
// parameters at a compile-time offset, so a low-bond exchange costs a handful of integer
// instructions and no branch: test the two spins, xor the byte offsets, read the rank
// table, read x from shared memory, add under the test's predicate.  The rank tables are
// kept pre-multiplied by the element size, so table values are byte offsets.
// ---------------------------------------------------------------------------------------
constexpr int BLK_XPAD = 128;        // a failed exchange may index up to 70 rows past a block

__shared__ uint32_t s_US[16 * 128];  // sizeof(element) * U[k][b1]   (K <= 15)
__shared__ uint32_t s_R0S[256];      // sizeof(element) * R0[b0]
__shared__ uint32_t s_hnext[2];      // dynamic schedule: blocks handed to this CTA

struct XSlot {                       // a cross bond in the current block
    const unsigned char *base;       // first row of the target block (flipped: its last row,
                                     // in the complement block; the target is base - offset)
    uint16_t wm, vm;                 // allowed iff (l ^ wm) & vm: bit p differs from bit q of h;
                                     // vm bit 15 (above every low position) marks a flipped target
    uint32_t kofs2;                  // byte offset of row k2 of s_US (k2 = k -+ 1)
};
constexpr uint16_t BLK_XFLIP = 0x8000u;

constexpr int BLK_HBI = HM_BLK_MAXB + 4 * HM_BLK_MAXC;   // high-exchange list with its padding

struct BlkMeta {                     // per-block data, double-buffered
    XSlot xs[HM_BLK_MAXC * 2 * HM_BLK_SX];
    // element index of the first row of each allowed high-exchange target block; class c
    // occupies [hs[c], he[c]) with hs[c] a multiple of 4, so four entries are one 16-byte load
    __align__(16) uint32_t hbi[BLK_HBI];
    int hs[HM_BLK_MAXC], he[HM_BLK_MAXC];
    uint32_t hv[2];
    uint32_t off, n, kofs, lwo;
    struct BlkMetaX *x;              // spin-flip / per-bond data of the block, or nullptr
};

// Per-block data that only spin-flip and per-bond plans use, in a shared-memory region of
// its own (allocated only for those plans, so the others keep the smaller footprint).
struct BlkMetaXF {
    // spin-flip basis: exchanges that move site N-1 lead out of the representatives; their
    // target is row n - 1 - r of the complement block, hbf[e] its last row, by class
    uint32_t hbf[HM_BLK_MAXB];
    int fs[HM_BLK_MAXC], fe[HM_BLK_MAXC];
    uint32_t hf[2];
};
struct BlkMetaX : BlkMetaXF {
    // per-bond plan (a spin-flip plan with classes allocates only the BlkMetaXF part):
    // coefficient of each entry of hbi and of hbf, integer (C_b, FP64 rows) and float (FP32 rows)
    long long hbc[BLK_HBI], hbfc[HM_BLK_MAXB];
    float hbcf[BLK_HBI], hbfcf[HM_BLK_MAXB];
};

// bits below position e of the 64-bit mask m
__device__ __forceinline__ int popc_below(uint64_t m, int e) {
    return e >= 64 ? __popcll(m) : __popcll(m & ((1ull << e) - 1ull));
}

// sum of the high-exchange gathers of class c for row r (the same low word in each target
// block), NH gathers in flight: four target offsets per 16-byte shared load (NH = 4), two per
// 8-byte load (NH = 2), or one at a time (NH = 1; fewest live registers).  PRED (NH = 4):
// the last round's loads past the class's run (padded to a multiple of four entries) are
// predicated off instead of taken one by one in a tail loop, so no gather waits for another.
// Which form is faster depends on the kernel's register allocation at 40 registers: the FP32
// rows predicate (N = 32 product 11.07 -> 10.16 ms), the FP64 rows of the sector product
// predicate with the values added in sequence (14.80 -> 14.69 ms), the FP64 spin-flip rows
// keep the tail loop (8.18 against 8.59 ms).
template <class Sv, int NH = 4, bool PRED = (sizeof(Sv) == 4), class G>
__device__ __forceinline__ Sv blk_high_sum(const BlkMeta &B, int c, const unsigned char *Xg, uint32_t r,
                                           const G &gx) {
    const int e0 = B.hs[c], e1 = B.he[c];
    Sv a = Sv(0);
    int e = e0;
    if constexpr (NH == 4) {
        const uint4 *h4 = reinterpret_cast<const uint4 *>(B.hbi);
        for (; PRED ? e < e1 : e + 4 <= e1; e += 4) {
            const uint4 t = h4[e >> 2];
            if constexpr (PRED && sizeof(Sv) == 8) {
                const uint32_t tt[4] = {t.x, t.y, t.z, t.w};
                Sv v[4];
#pragma unroll
                for (int i = 0; i < 4; ++i) v[i] = e + i < e1 ? gx(Xg + (size_t)(tt[i] + r) * sizeof(Sv)) : Sv(0);
#pragma unroll
                for (int i = 0; i < 4; ++i) a += v[i];
            } else {
                const Sv v0 = gx(Xg + (size_t)(t.x + r) * sizeof(Sv));
                const Sv v1 = !PRED || e + 1 < e1 ? gx(Xg + (size_t)(t.y + r) * sizeof(Sv)) : Sv(0);
                const Sv v2 = !PRED || e + 2 < e1 ? gx(Xg + (size_t)(t.z + r) * sizeof(Sv)) : Sv(0);
                const Sv v3 = !PRED || e + 3 < e1 ? gx(Xg + (size_t)(t.w + r) * sizeof(Sv)) : Sv(0);
                a += (v0 + v1) + (v2 + v3);
            }
        }
    } else if constexpr (NH == 2) {
        const uint2 *h2 = reinterpret_cast<const uint2 *>(B.hbi);
        for (; e + 2 <= e1; e += 2) {
            const uint2 t = h2[e >> 1];
            a += gx(Xg + (size_t)(t.x + r) * sizeof(Sv)) + gx(Xg + (size_t)(t.y + r) * sizeof(Sv));
        }
    }
    if constexpr (!(NH == 4 && PRED))
        for (; e < e1; ++e) a += gx(Xg + (size_t)(B.hbi[e] + r) * sizeof(Sv));
    return a;
}

// spin-flip basis: sum of the flipped high-exchange gathers of class c for row r (row
// n - 1 - r of each complement block), before the parity sign
template <class Sv, class G>
__device__ __forceinline__ Sv blk_flip_sum(const BlkMeta &B, int c, const unsigned char *Xg, uint32_t r,
                                           const G &gx) {
    Sv a = Sv(0);
    const BlkMetaX &X = *B.x;
    for (int e = X.fs[c]; e < X.fe[c]; ++e) a += gx(Xg + (size_t)(X.hbf[e] - r) * sizeof(Sv));
    return a;
}

// ---- per-bond rows: y_i = g0 x_i + sum over allowed exchanges of h_b (x_i - x_t) ----------
// fixed-point rows: exact int128 sum of C_b (x_i - x_t) (|C_b| <= 2^61, |x_i - x_t| < 2^54,
// at most 64 terms and C0 x_i: below 2^123); FP32 rows: float multiply-adds
template <class Sv> struct PbAcc { using T = __int128; };
template <> struct PbAcc<float> { using T = float; };
__device__ __forceinline__ __int128 pb_mac(long long C, float, int64_t d, __int128 a) { return a + (__int128)C * d; }
__device__ __forceinline__ float pb_mac(long long, float Cf, float d, float a) { return fmaf(Cf, d, a); }

__device__ __forceinline__ double i128_to_double(__int128 v) {
    const long long hi = (long long)(v >> 64);
    const unsigned long long lo = (unsigned long long)v;
    return (double)hi * 18446744073709551616.0 + (double)lo;
}

// high exchanges of a per-bond plan (class 0 lists), four gathers at a time; flipped
// targets carry the parity
template <class Sv, class G>
__device__ __forceinline__ typename PbAcc<Sv>::T blk_high_pb(const BlkParams &P, const BlkMeta &B,
                                                             const unsigned char *Xg, uint32_t r, const G &gx,
                                                             Sv xo, typename PbAcc<Sv>::T a) {
    const BlkMetaX &X = *B.x;
    const int e1 = B.he[0];
    const uint4 *h4 = reinterpret_cast<const uint4 *>(B.hbi);
    int e = B.hs[0];
    for (; e + 4 <= e1; e += 4) {
        const uint4 t = h4[e >> 2];
        const Sv v0 = gx(Xg + (size_t)(t.x + r) * sizeof(Sv)), v1 = gx(Xg + (size_t)(t.y + r) * sizeof(Sv));
        const Sv v2 = gx(Xg + (size_t)(t.z + r) * sizeof(Sv)), v3 = gx(Xg + (size_t)(t.w + r) * sizeof(Sv));
        a = pb_mac(X.hbc[e], X.hbcf[e], xo - v0, a);
        a = pb_mac(X.hbc[e + 1], X.hbcf[e + 1], xo - v1, a);
        a = pb_mac(X.hbc[e + 2], X.hbcf[e + 2], xo - v2, a);
        a = pb_mac(X.hbc[e + 3], X.hbcf[e + 3], xo - v3, a);
    }
    for (; e < e1; ++e) a = pb_mac(X.hbc[e], X.hbcf[e], xo - gx(Xg + (size_t)(B.hbi[e] + r) * sizeof(Sv)), a);
    for (int f = X.fs[0]; f < X.fe[0]; ++f) {
        const Sv v = gx(Xg + (size_t)(X.hbf[f] - r) * sizeof(Sv));
        a = pb_mac(X.hbfc[f], X.hbfcf[f], xo - (P.par < 0 ? -v : v), a);
    }
    return a;
}

__device__ __forceinline__ uint32_t us_at(uint32_t byte_off) {
    return *(const uint32_t *)((const unsigned char *)s_US + byte_off);
}
__device__ __forceinline__ uint32_t r0s_at(uint32_t byte_off) {
    return *(const uint32_t *)((const unsigned char *)s_R0S + byte_off);
}

// dynamic shared memory of the sweep: staged rows (+ pad elements) | 2 BlkMeta
__host__ __device__ __forceinline__ size_t blk_row_xs_bytes(const BlkParams &P, int esize, int pad) {
    return al16(((size_t)P.max_block + pad) * esize);
}
// bytes of one BlkMetaX copy the plan uses (0: none)
__host__ __device__ __forceinline__ size_t blk_x_bytes(const BlkParams &P) {
    return P.perbond ? al16(sizeof(BlkMetaX)) : P.par ? al16(sizeof(BlkMetaXF)) : 0;
}
// the table C (binomials D(p, c), p <= N, c <= A) staged in shared memory when it takes at
// most 4 KB (2.2 KB for N = 32, M = 0): the block set-up's offsets off(h) read it in a loop
// over the high word's ones, a chain of dependent-issue loads between two CTA barriers
__host__ __device__ __forceinline__ size_t blk_c_bytes(const BlkParams &P) {
    const size_t b = (size_t)(P.N + 1) * (P.A + 1) * sizeof(uint32_t);
    return b <= 4096 ? al16(b) : 0;
}

__host__ __device__ __forceinline__ size_t blk_row_smem_bytes(const BlkParams &P, int esize, int pad) {
    return blk_row_xs_bytes(P, esize, pad) + 2 * al16(sizeof(BlkMeta)) + 2 * blk_x_bytes(P) + blk_c_bytes(P);
}

__device__ __forceinline__ bool blk_h_valid(const BlkParams &P, uint32_t h) {
    const int k = P.A - __popc(h);
    return k >= 0 && k <= P.K;
}

// block of schedule position c: h = c, or (P.rot > 0) c with its low rot bits moved to the
// top of the high word, so that the top rot high sites vary fastest along the schedule
__device__ __forceinline__ uint32_t blk_order(const BlkParams &P, uint32_t c) {
    if (!P.rot) return c;
    const int R = P.rot;
    return (c >> R) | ((c & ((1u << R) - 1u)) << (P.H - R));
}

// next block of the dynamic schedule (positions handed out in increasing order; without
// rotation that is increasing h, i.e. increasing row index); >= nH when none is left
__device__ __forceinline__ uint32_t blk_fetch(const BlkParams &P, unsigned *sched, uint32_t nH) {
    uint32_t c, h;
    do {
        c = atomicAdd(&sched[0], 1u);
        h = c < nH ? blk_order(P, c) : c;
    } while (c < nH && !blk_h_valid(P, h));
    return h;
}

// gathers: element at a byte address of the vector
// read-only global loads (through the non-coherent path; the data do not change while a
// kernel runs)
__device__ __forceinline__ long long ldg_s64(const void *p) { return __ldg((const long long *)p); }
__device__ __forceinline__ uint4 ldg_v4(const uint4 *p) { return __ldg(p); }

struct GFix {                        // fixed-point copy
    __device__ __forceinline__ int64_t operator()(const unsigned char *p) const {
        return (int64_t)ldg_s64(p);
    }
};
struct GF64 {                        // binary64, converted to fixed point (exponent E)
    int E;
    __device__ __forceinline__ int64_t operator()(const unsigned char *p) const {
        return ef::fix_from_bits(__ldg((const unsigned long long *)p), E);
    }
};
struct GF32 {
    __device__ __forceinline__ float operator()(const unsigned char *p) const { return __ldg((const float *)p); }
};

#define HM_XS(off_) (*(const Sv *)(Xsb + (off_)))
#define HM_L0(s) { const uint32_t z_ = l ^ (l >> P.ld[c][0][s]);                                  \
        const uint32_t v_ = r0s_at((l4 ^ P.lxa[c][0][s]) & 0x3FCu);                               \
        if (z_ & P.lvm[c][0][s]) a += HM_XS(R1own + v_); }
#define HM_L1(s) { const uint32_t z_ = l ^ (l >> P.ld[c][1][s]);                                  \
        const uint32_t v_ = us_at(lh4k ^ P.lxb[c][1][s]);                                          \
        if (z_ & P.lvm[c][1][s]) a += HM_XS(R0own + v_); }
#define HM_L2(s) { const uint32_t z_ = l ^ (l >> P.ld[c][2][s]);                                  \
        const uint32_t v_ = us_at(lh4k ^ P.lxb[c][2][s]) + r0s_at((l4 ^ P.lxa[c][2][s]) & 0x3FCu); \
        if (z_ & P.lvm[c][2][s]) a += HM_XS(v_); }
#define HM_LG(g) m += __popc((l ^ (l >> P.lgd[c][g])) & P.lgm[c][g]);
#define HM_XADD(v_) { if (x_.vm & BLK_XFLIP) { const Sv t_ = gx(x_.base - (v_)); a += P.par < 0 ? -t_ : t_; } \
        else a += gx(x_.base + (v_)); ++m; }
#define HM_X0(s) { const XSlot x_ = B.xs[(2 * c) * HM_BLK_SX + (s)];                              \
        const uint32_t v_ = us_at(lh4 | x_.kofs2) + r0s_at((l4 ^ P.xxa[c][0][s]) & 0x3FCu);        \
        if ((l ^ x_.wm) & x_.vm) HM_XADD(v_) }
#define HM_X1(s) { const XSlot x_ = B.xs[(2 * c + 1) * HM_BLK_SX + (s)];                          \
        const uint32_t v_ = us_at((lh4 ^ P.xxa[c][1][s]) | x_.kofs2) + R0own;                      \
        if ((l ^ x_.wm) & x_.vm) HM_XADD(v_) }
// a switch entering an unrolled run of slots n-1, ..., 0
#define HM_RUN16(M) case 16: M(15) [[fallthrough]]; case 15: M(14) [[fallthrough]]; case 14: M(13) [[fallthrough]]; \
    case 13: M(12) [[fallthrough]]; case 12: M(11) [[fallthrough]]; case 11: M(10) [[fallthrough]];                \
    case 10: M(9) [[fallthrough]]; case 9: M(8) [[fallthrough]]; HM_RUN8(M)
#define HM_RUN8(M) case 8: M(7) [[fallthrough]]; case 7: M(6) [[fallthrough]]; HM_RUN6(M)
#define HM_RUN6(M) case 6: M(5) [[fallthrough]]; case 5: M(4) [[fallthrough]]; case 4: M(3) [[fallthrough]]; \
    case 3: M(2) [[fallthrough]]; case 2: M(1) [[fallthrough]]; case 1: M(0) [[fallthrough]]; default: break;

// Row policy: Row::sums(P, B, Xsb, Xg, l, r, gx, acc, cnt) sets, for row r (low word l) of
// the current block, acc[c] = sum of x over the allowed exchanges of class c and cnt[c]
// = their number.  RowGeneric reads the bond slots from the parameters; the kernels
// specialised at run time (jit.cu) bring a policy with the slots written out.
//
// A policy also says how many pad elements follow the staged rows (kPad), whether the
// cross slots index rows k-1, k, k+1 of a per-block copy of US (kRelUS) or US itself,
// and has two hooks: stage<Sv>(P) at kernel start (all threads, before the first
// barrier, with the dynamic shared base; s_R0S is being written in the same phase and
// may not be read) and
// block<Sv>(P, k) once per block between the block setup and the rows (all threads).
template <int NC>
struct RowGeneric {
static constexpr int kPad = BLK_XPAD;
static constexpr bool kRelUS = false;
static constexpr bool kPerBond = false;      // per-bond plans run only specialised (jit.cu)
static constexpr bool kBC = false;           // bond-correlation rows (jit.cu) neither
template <class Sv>
static __device__ __forceinline__ void stage(const BlkParams &P, unsigned char *) {
    const uint16_t *Ug = (const uint16_t *)((const unsigned char *)P.tab + P.off_U);
    const int nU = (P.K + 1) * P.nb1;
    for (int i = threadIdx.x; i < nU; i += BLK_NT) s_US[i] = (uint32_t)Ug[i] * (uint32_t)sizeof(Sv);
}
template <class Sv>
static __device__ __forceinline__ void block(const BlkParams &, uint32_t) {}
template <class Sv, class G>
static __device__ __forceinline__ void sums(const BlkParams &P, const BlkMeta &B, const unsigned char *Xsb,
                                            const unsigned char *Xg, uint32_t l, uint32_t r, const G &gx, Sv xo,
                                            Sv *acc, int *cnt) {
    (void)xo;
    const uint32_t l4 = l << 2, lh4 = (l >> 8) << 2, lh4k = lh4 | B.kofs;
    const uint32_t R0own = r0s_at(l4 & 0x3FCu), R1own = us_at(lh4k);
#pragma unroll
    for (int c = 0; c < NC; ++c) {
        Sv a = Sv(0);
        int m = 0;
        switch (P.ln[c][0]) { HM_RUN16(HM_L0) }
        switch (P.ln[c][1]) { HM_RUN16(HM_L1) }
        switch (P.ln[c][2]) { HM_RUN16(HM_L2) }
        switch (P.lgn[c]) { HM_RUN6(HM_LG) }
        switch (P.xn[c][0]) { HM_RUN8(HM_X0) }
        switch (P.xn[c][1]) { HM_RUN8(HM_X1) }
        // exchanges among the high positions: the same low word in another block
        a += blk_high_sum<Sv>(B, c, Xg, r, gx);
        if (P.par) {
            const Sv f = blk_flip_sum<Sv>(B, c, Xg, r, gx);
            a += P.par < 0 ? -f : f;
        }
        acc[c] = a;
        cnt[c] = m + (B.he[c] - B.hs[c]) + (P.par ? B.x->fe[c] - B.x->fs[c] : 0);
    }
}
};
#undef HM_XS
#undef HM_L0
#undef HM_L1
#undef HM_L2
#undef HM_LG
#undef HM_X0
#undef HM_X1
#undef HM_XADD

// Every block of the sector through rowf(off, r, x_r, acc, cnt, pref(off + r)) once
// (pref loads what the row needs besides x, issued before the hop sums).  X: the vector as
// gx reads it (element size sizeof(Sv)).  DYN: blocks handed out in increasing order by
// the counter pair sched (zero on entry, zero again on exit), so the CTAs sweep the
// vector together and the targets of nearby exchanges are still in L2; otherwise a
// static round robin.  After the rows of a block every thread calls endf(it); one thread
// then calls flushf(h, it) once the whole CTA is past endf(it), so per-block reductions
// come out the same whichever CTA ran the block.  All threads of the CTA must call it.
template <class Sv, int NC, bool DYN, class Row, class G, class PrefF, class RowF, class EndF, class FlushF>
__device__ __forceinline__ void blk_sweep(const BlkParams &P, const unsigned char *X, const G &gx, unsigned *sched,
                                          PrefF &&pref, RowF &&rowf, EndF &&endf, FlushF &&flushf) {
    extern __shared__ __align__(16) unsigned char smem[];
    const unsigned char *Xsb = smem;
    Sv *Xs = (Sv *)smem;
    BlkMeta *meta = (BlkMeta *)(smem + blk_row_xs_bytes(P, sizeof(Sv), Row::kPad));
    unsigned char *metax = blk_x_bytes(P) ? (unsigned char *)meta + 2 * al16(sizeof(BlkMeta)) : nullptr;
    const int tid = threadIdx.x;
    const uint32_t *Cg = (const uint32_t *)((const unsigned char *)P.tab + P.off_C);
    {
        const uint8_t *R0g = (const uint8_t *)P.tab + P.off_R0;
        for (int i = tid; i < 256; i += BLK_NT) s_R0S[i] = (uint32_t)R0g[i] * (uint32_t)sizeof(Sv);
        Row::template stage<Sv>(P, smem);
        if (blk_c_bytes(P)) {
            uint32_t *Cs = (uint32_t *)(smem + blk_row_xs_bytes(P, sizeof(Sv), Row::kPad) + 2 * al16(sizeof(BlkMeta)) +
                                        2 * blk_x_bytes(P));
            for (int i = tid; i < (P.N + 1) * (P.A + 1); i += BLK_NT) Cs[i] = Cg[i];
            Cg = Cs;
        }
    }
    BlkTabs tb;
    tb.U = nullptr; tb.R0 = nullptr; tb.C = Cg;
    // spin-flip basis: only the representatives, the blocks whose site N-1 is up
    const uint32_t nH = 1u << (P.H - (P.par ? 1 : 0));
    if (DYN && tid == 0) s_hnext[0] = blk_fetch(P, sched, nH);
    __syncthreads();
    uint32_t hs = blockIdx.x, h_prev = 0u;
    int it_prev = -1;
    for (int it = 0;; ++it) {
        uint32_t h;
        if (DYN) {
            h = s_hnext[it & 1];
        } else {
            h = hs;
            while (h < nH && !blk_h_valid(P, h)) h += gridDim.x;
            hs = h + gridDim.x;
        }
        if (h >= nH) break;
        BlkMeta &B = meta[it & 1];
        BlkMetaX *BX = metax ? (BlkMetaX *)(metax + (it & 1) * blk_x_bytes(P)) : nullptr;
        const int k = P.A - __popc(h);
        // setup 1: targets of the high and cross exchanges, own offset, next block
        if (DYN && tid == 0) s_hnext[(it + 1) & 1] = blk_fetch(P, sched, nH);
        uint32_t hidx = 0u;
        bool hval = false, hflip = false;
        if (tid < P.nhb) {
            const int p = P.hb_p[tid], q = P.hb_q[tid];
            const bool ok = (((h >> p) ^ (h >> q)) & 1u) != 0u;
            const uint32_t h2 = h ^ ((1u << p) | (1u << q));
            if (ok && P.par && q == P.H - 1) {     // site N-1 flips up: the complement block
                hflip = true;
                hidx = blk_off(P, tb, ~h2 & ((1u << P.H) - 1u), P.K - k) + Cg[P.K * (P.A + 1) + k] - 1u;
            } else if (ok) {
                hval = true;
                hidx = blk_off(P, tb, h2, k);
            }
        }
        if (tid < 64) {
            const unsigned bal = __ballot_sync(0xffffffffu, hval), balf = __ballot_sync(0xffffffffu, hflip);
            if ((tid & 31) == 0) {
                B.hv[tid >> 5] = bal;
                if (BX) BX->hf[tid >> 5] = balf;
            }
        }
        if (tid >= 64 && tid < 64 + P.nxf) {
            const int e = tid - 64, p = P.xf_p[e], q = P.xf_q[e];
            const uint32_t bq = (h >> q) & 1u;
            const int k2 = k + (bq ? 1 : -1);
            const bool ok = k2 >= 0 && k2 <= P.K;
            const bool fl = ok && P.par && q == P.H - 1;   // site N-1 flips up: complement block
            XSlot xs;
            xs.base = !ok ? X
                      : fl ? X + (size_t)(blk_off(P, tb, ~(h ^ (1u << q)) & ((1u << P.H) - 1u), P.K - k2) +
                                          Cg[P.K * (P.A + 1) + k2] - 1u) * sizeof(Sv)
                           : X + (size_t)blk_off(P, tb, h ^ (1u << q), k2) * sizeof(Sv);
            xs.wm = (uint16_t)(bq << p);
            xs.vm = (uint16_t)(ok ? (1u << p) | (fl ? BLK_XFLIP : 0u) : 0u);
            xs.kofs2 = ok ? (uint32_t)(Row::kRelUS ? k2 - k + 1 : k2) << P.kshift : 0u;
            B.xs[P.xf_dst[e]] = xs;
        }
        if (tid == 128) {
            B.x = BX;
            B.off = blk_off(P, tb, h, k);
            B.n = Cg[P.K * (P.A + 1) + k];
            B.kofs = (uint32_t)k << P.kshift;
            B.lwo = (uint32_t)P.lwoff[k];
        }
        __syncthreads();
        if (tid == BLK_NT - 1 && it_prev >= 0) flushf(h_prev, it_prev);
        // setup 2: compact the allowed high exchanges by class, each class's run padded to a
        // multiple of 4 entries; stage the block's x
        if (P.bcmode) {                              // bond correlations: high bond j at hbi[j]
            if (tid < P.nhb) B.hbi[tid] = hval ? hidx : 0xFFFFFFFFu;
        } else if (hval || hflip || tid < HM_BLK_MAXC) {
            const uint64_t hm = ((uint64_t)B.hv[1] << 32) | B.hv[0];
            const uint64_t fm = BX ? ((uint64_t)BX->hf[1] << 32) | BX->hf[0] : 0ull;
            int start = 0;                           // padded start of the class
            for (int c = 0; c < HM_BLK_MAXC; ++c) {
                const int b0 = popc_below(hm, P.hb_start[c]), b1 = popc_below(hm, P.hb_start[c + 1]);
                const int f0 = popc_below(fm, P.hb_start[c]), f1 = popc_below(fm, P.hb_start[c + 1]);
                if (tid >= P.hb_start[c] && tid < P.hb_start[c + 1]) {
                    const float cf = P.perbond ? (float)ldexp((double)P.pb_hc[tid], -P.pb_s) : 0.0f;
                    if (hval) {
                        B.hbi[start + popc_below(hm, tid) - b0] = hidx;
                        if (P.perbond) {
                            BX->hbc[start + popc_below(hm, tid) - b0] = P.pb_hc[tid];
                            BX->hbcf[start + popc_below(hm, tid) - b0] = cf;
                        }
                    }
                    if (hflip) {
                        BX->hbf[popc_below(fm, tid)] = hidx;
                        if (P.perbond) { BX->hbfc[popc_below(fm, tid)] = P.pb_hc[tid]; BX->hbfcf[popc_below(fm, tid)] = cf; }
                    }
                }
                if (tid == c) {
                    B.hs[c] = start;
                    B.he[c] = start + (b1 - b0);
                    if (BX) { BX->fs[c] = f0; BX->fe[c] = f1; }
                }
                start += (b1 - b0 + 3) & ~3;
            }
        }
        const uint32_t off = B.off, n = B.n;
        for (uint32_t r = tid; r < n; r += BLK_NT) Xs[r] = gx(X + (size_t)(off + r) * sizeof(Sv));
        Row::template block<Sv>(P, (uint32_t)k);
        __syncthreads();
        const uint16_t *lw = P.lw + B.lwo;
        uint32_t l_next = tid < n ? (uint32_t)__ldg(lw + tid) : 0u;
        for (uint32_t r = tid; r < n; r += BLK_NT) {
            const uint32_t l = l_next;                     // the list word one row ahead
            if (r + BLK_NT < n) l_next = (uint32_t)__ldg(lw + r + BLK_NT);
            const auto pv = pref(off + r);                 // the row's other operand, ahead of the sums
            const Sv xo = Xs[r];
            if constexpr (Row::kBC) {
                rowf(off, r, xo, pv, B, Xsb, l);
            } else if constexpr (Row::kPerBond) {
                rowf(off, r, xo, Row::template sums_pb<Sv>(P, B, Xsb, X, l, r, gx, xo), pv);
            } else {
                Sv acc[NC];
                int cnt[NC];
                Row::template sums<Sv>(P, B, Xsb, X, l, r, gx, xo, acc, cnt);
                rowf(off, r, xo, acc, cnt, pv);
            }
        }
        endf(it);
        h_prev = h;
        it_prev = it;
    }
    __syncthreads();
    if (tid == BLK_NT - 1 && it_prev >= 0) flushf(h_prev, it_prev);
    if (DYN && tid == 0) {
        if (atomicAdd(&sched[1], 1u) == gridDim.x - 1) {   // every CTA is past its last fetch
            sched[0] = 0u;
            sched[1] = 0u;
        }
    }
}

// s 2^k as binary64 bits, rounded to nearest even: the conversion unit's correctly rounded
// int64 -> binary64 conversion with its exponent field moved by k, exact while the result
// is a normal number; otherwise (zero, underflow, overflow) the integer rounding of
// ef::bits_from_int.  Both give the same bits wherever both apply; this one keeps about
// twenty integer instructions a row off the integer pipe.
__device__ __forceinline__ unsigned long long blk_bits_pow2(int64_t s, int k) {
    const unsigned long long b = ef::d2u(__ll2double_rn((long long)s));
    const int e = (int)((b >> 52) & 0x7FFu) + k;
    if (s != 0 && e >= 1 && e <= 2046) return b + ((unsigned long long)(long long)k << 52);
    return ef::bits_from_int(s, k);
}

// T_c = 2 acc_c + (ntot_c - 2 cnt_c) x_i: the class sum of Eq. (E-2-1) rows in units of
// -J_c / 4 (s = 1/2: s^z s^z = +-1/4, exchange element 1/2)
template <int NC>
__device__ __forceinline__ void blk_classes(const BlkParams &P, const int64_t *acc, const int *cnt, int64_t Xo,
                                            int64_t *T) {
#pragma unroll
    for (int c = 0; c < NC; ++c) T[c] = 2 * acc[c] + (int64_t)(P.ntot[c] - 2 * cnt[c]) * Xo;
}

// y (binary64 bits) of a row from its class sums; u = unit exponent of the fixed point.
// Integer-ratio classes with a power-of-two g0 round the exact integer once.
template <int NC, int IRM = -1>       // IRM: integer ratios known at compile time (1 / 0), or -1
__device__ __forceinline__ unsigned long long blk_y_bits(const BlkParams &P, const int64_t *T, int u, int64_t *Tsum) {
    if (IRM == 1 || (IRM < 0 && P.iratio)) {
        int64_t s = 0;
#pragma unroll
        for (int c = 0; c < NC; ++c) s += (int64_t)P.Kc[c] * T[c];
        *Tsum = s;
        if (P.g0_pow2) return blk_bits_pow2(s, u + P.g0_exp);
        const ef::df t = ef::df_from_fix(s, u + 1022 + ef::FIX_BITS, 0, 0);
        return ef::bits_from_df(ef::df_mul(t, ef::df{P.g0_hi, P.g0_lo}), 0);
    }
    *Tsum = 0;
    ef::df y{0.0f, 0.0f};
#pragma unroll
    for (int c = 0; c < NC; ++c)
        y = ef::df_add(y, ef::df_mul(ef::df_from_fix(T[c], u + 1022 + ef::FIX_BITS, 0, 0), ef::df{P.g_hi[c], P.g_lo[c]}));
    return ef::bits_from_df(y, 0);
}

template <int NC>
__device__ __forceinline__ float blk_y_f32(const BlkParams &P, const float *acc, const int *cnt, float xo) {
    float y = 0.0f;
#pragma unroll
    for (int c = 0; c < NC; ++c) y += P.gq[c] * (2.0f * acc[c] + (float)(P.ntot[c] - 2 * cnt[c]) * xo);
    return y;
}

// ---------------------------------------------------------------------------------------
// y = H x (matvec API)
// ---------------------------------------------------------------------------------------
template <class T, int NC, class Row>
__device__ __forceinline__ void matvec_body(const BlkParams &P, const T *__restrict__ x, T *__restrict__ y,
                                            const int *__restrict__ Eptr) {
    if constexpr (sizeof(T) == 8) {
        const int E = Eptr ? *Eptr : 0;
        const int u = E - 1022 - ef::FIX_BITS;
        unsigned long long *yb = (unsigned long long *)y;
        if constexpr (Row::kPerBond) {
            const double sy = ef::pow2d(u - P.pb_s);
            blk_sweep<int64_t, NC, false, Row>(P, (const unsigned char *)x, GF64{E}, nullptr, [](uint32_t) { return 0; },
                                          [&](uint32_t off, uint32_t r, int64_t xo, __int128 sv, int) {
                                              const __int128 t = (__int128)P.pb_c0 * xo + sv;
                                              yb[off + r] = ef::d2u(i128_to_double(t) * sy);
                                          },
                                          [](int) {}, [](uint32_t, int) {});
        } else {
            blk_sweep<int64_t, NC, false, Row>(P, (const unsigned char *)x, GF64{E}, nullptr, [](uint32_t) { return 0; },
                                          [&](uint32_t off, uint32_t r, int64_t xo, const int64_t *acc, const int *cnt, int) {
                                              int64_t Tc[NC], ts;
                                              blk_classes<NC>(P, acc, cnt, xo, Tc);
                                              yb[off + r] = blk_y_bits<NC>(P, Tc, u, &ts);
                                          },
                                          [](int) {}, [](uint32_t, int) {});
        }
    } else {
        if constexpr (Row::kPerBond) {
            blk_sweep<float, NC, false, Row>(P, (const unsigned char *)x, GF32{}, nullptr, [](uint32_t) { return 0; },
                                        [&](uint32_t off, uint32_t r, float xo, float sv, int) {
                                            y[off + r] = fmaf((float)P.pb_g0, xo, sv);
                                        },
                                        [](int) {}, [](uint32_t, int) {});
        } else {
            blk_sweep<float, NC, false, Row>(P, (const unsigned char *)x, GF32{}, nullptr, [](uint32_t) { return 0; },
                                        [&](uint32_t off, uint32_t r, float xo, const float *acc, const int *cnt, int) {
                                            y[off + r] = blk_y_f32<NC>(P, acc, cnt, xo);
                                        },
                                        [](int) {}, [](uint32_t, int) {});
        }
    }
}

// ---------------------------------------------------------------------------------------
// Lanczos, FP64: y = H q_cur from the fixed-point copy Xc of q_cur (every gather an
// integer load), written as binary64 to Y; the exact integer dot q.y gives alpha
// (with q.q_prev from the fixed-point copy kernel) without re-reading y.
// ---------------------------------------------------------------------------------------

// per-warp partial sums of the current and previous block (blk_sweep's endf / flushf)
__shared__ double s_wpart[2][BLK_NT / 32][1];

__device__ __forceinline__ double warp_sum(double v) {
    for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
    return v;
}

// part[h] = (q . H q) over the rows of block h, in true units; entries of blocks that do
// not exist stay as they are.
// SPLIT = 1 / 2: the two passes of the split product (integer-ratio classes with a power-of-
// two unit g0).  Pass 1 (plan of the near bonds) stores each row's exact integer
// sum_c K_c T_c in Y; pass 2 (plan of the far bonds, rotated block order) adds its own,
// rounds the total once to binary64 in place and forms q.Hq from it.  The total is the same
// integer the single pass forms, so both give the same bits.
template <int NC, bool IR, class Row, int SPLIT = 0>
__device__ __forceinline__ void lz64_body(const BlkParams &P, const long long *__restrict__ Xc,
                                          unsigned long long *__restrict__ Y, LzScalars *S, int pc,
                                          double *__restrict__ part) {
    if (S->done) return;
    if constexpr (SPLIT != 0) {
        static_assert(IR && !Row::kPerBond, "the split product needs integer-ratio classes");
        const int E = S->emax[pc];
        const int u = E - 1022 - ef::FIX_BITS;
        auto tsum = [&](int64_t xo, const int64_t *acc, const int *cnt) {
            int64_t Tc[NC];
            blk_classes<NC>(P, acc, cnt, xo, Tc);
            int64_t s = 0;
#pragma unroll
            for (int c = 0; c < NC; ++c) s += (int64_t)P.Kc[c] * Tc[c];
            return s;
        };
        if constexpr (SPLIT == 1) {
            blk_sweep<int64_t, NC, true, Row>(
                P, (const unsigned char *)Xc, GFix{}, S->sched, [](uint32_t) { return 0; },
                [&](uint32_t off, uint32_t r, int64_t xo, const int64_t *acc, const int *cnt, int) {
                    __stcs(Y + off + r, (unsigned long long)tsum(xo, acc, cnt));
                },
                [](int) {}, [](uint32_t, int) {});
        } else {
            __int128 d1 = 0;
            blk_sweep<int64_t, NC, true, Row>(
                P, (const unsigned char *)Xc, GFix{}, S->sched,
                [&](uint32_t i) { return (long long)__ldcs(Y + i); },
                [&](uint32_t off, uint32_t r, int64_t xo, const int64_t *acc, const int *cnt, long long sa) {
                    const int64_t s = (int64_t)sa + tsum(xo, acc, cnt);
                    __stcs(Y + off + r, blk_bits_pow2(s, u + P.g0_exp));
                    d1 += (__int128)xo * s;
                },
                [&](int it) {
                    const double q_y = ldexp(i128_to_double(d1) * P.g0, 2 * u);
                    d1 = 0;
                    const double a = warp_sum(q_y);
                    if ((threadIdx.x & 31) == 0) s_wpart[it & 1][threadIdx.x >> 5][0] = a;
                },
                [&](uint32_t h, int it) {
                    double a = 0.0;
                    for (int w = 0; w < BLK_NT / 32; ++w) a += s_wpart[it & 1][w][0];
                    part[h] = a;
                });
        }
        return;
    }
    const int E = S->emax[pc];
    const int u = E - 1022 - ef::FIX_BITS;
    __int128 d1 = 0;
    ef::df d1f{0.0f, 0.0f};
    // row value: exact class sums, or (per-bond plan) one binary64 sum of h_b (x_i - x_t).
    // Integer ratios: s = sum_c K_c T_c = 2 sum_c K_c acc_c + (sum_c K_c (n_c - 2 cnt_c)) x_i,
    // one exact integer (|K_c| <= 64 and sum_c |K_c| n_c < 334, so the second factor is a
    // small int and every partial stays below 2^63), rounded once to binary64
    auto rowc = [&](uint32_t off, uint32_t r, int64_t xo, const int64_t *acc, const int *cnt, int) {
        if constexpr (IR) {
            int64_t a = 0;
            int m = 0;
#pragma unroll
            for (int c = 0; c < NC; ++c) {
                a += (int64_t)P.Kc[c] * acc[c];
                m += P.Kc[c] * (P.ntot[c] - 2 * cnt[c]);
            }
            const int64_t ts = 2 * a + (int64_t)m * xo;
            unsigned long long yb;
            if (P.g0_pow2) {
                yb = blk_bits_pow2(ts, u + P.g0_exp);
            } else {
                const ef::df t = ef::df_from_fix(ts, u + 1022 + ef::FIX_BITS, 0, 0);
                yb = ef::bits_from_df(ef::df_mul(t, ef::df{P.g0_hi, P.g0_lo}), 0);
            }
            __stcs(Y + off + r, yb);
            d1 += (__int128)xo * ts;
        } else {
            int64_t Tc[NC], ts;
            blk_classes<NC>(P, acc, cnt, xo, Tc);
            const unsigned long long yb = blk_y_bits<NC, 0>(P, Tc, u, &ts);
            __stcs(Y + off + r, yb);
            d1f = ef::df_add(d1f, ef::df_mul(ef::df_from_fix(xo, E, 0, E - 1023), ef::df_from_bits(yb, E - 1023)));
        }
    };
    const double sy = ef::pow2d(u - P.pb_s);
    auto rowb = [&](uint32_t off, uint32_t r, int64_t xo, __int128 sv, int) {
        const __int128 t = (__int128)P.pb_c0 * xo + sv;
        const unsigned long long yb = ef::d2u(i128_to_double(t) * sy);
        __stcs(Y + off + r, yb);
        d1f = ef::df_add(d1f, ef::df_mul(ef::df_from_fix(xo, E, 0, E - 1023), ef::df_from_bits(yb, E - 1023)));
    };
    auto endf = [&](int it) {
            // true units: q.y = g0 2^(2u) sum X Tsum (integer ratios) or the double-float
            // sum scaled back by 2^(2(E-1023))
            const double q_y = IR && !Row::kPerBond ? ldexp(i128_to_double(d1) * P.g0, 2 * u)
                                                    : ldexp((double)d1f.hi + (double)d1f.lo, 2 * (E - 1023));
            d1 = 0; d1f = ef::df{0.0f, 0.0f};
            const double a = warp_sum(q_y);
            if ((threadIdx.x & 31) == 0) s_wpart[it & 1][threadIdx.x >> 5][0] = a;
        };
    auto flushf = [&](uint32_t h, int it) {
            double a = 0.0;
            for (int w = 0; w < BLK_NT / 32; ++w) a += s_wpart[it & 1][w][0];
            part[h] = a;
        };
    if constexpr (Row::kPerBond)
        blk_sweep<int64_t, NC, true, Row>(P, (const unsigned char *)Xc, GFix{}, S->sched, [](uint32_t) { return 0; },
                                          rowb, endf, flushf);
    else
        blk_sweep<int64_t, NC, true, Row>(P, (const unsigned char *)Xc, GFix{}, S->sched, [](uint32_t) { return 0; },
                                          rowc, endf, flushf);
}

// ---------------------------------------------------------------------------------------
// Lanczos, FP32: u = sigma H q - gamma q_prev over q_prev, dot in double-float
// ---------------------------------------------------------------------------------------
// part[h] = (sigma q . u) over the rows of block h
template <int NC, class Row>
__device__ __forceinline__ void lz32_body(const BlkParams &P, const float *__restrict__ qc, float *__restrict__ qp,
                                          LzScalars *S, double *__restrict__ part) {
    if (S->done) return;
    const float sig = (float)S->sigma_cur, gam = (float)(S->beta_prev * S->sigma_prev);
    ef::df dot{0.0f, 0.0f};
    auto pref = [&](uint32_t i) { return qp[i]; };
    auto rowu = [&](uint32_t off, uint32_t r, float xo, float hv, float qpr) {
        const float uu = sig * hv - gam * qpr;
        qp[off + r] = uu;
        dot = ef::df_add(dot, ef::two_prod(sig * xo, uu));
    };
    auto endf = [&](int it) {
        const double a = warp_sum((double)dot.hi + (double)dot.lo);
        dot = ef::df{0.0f, 0.0f};
        if ((threadIdx.x & 31) == 0) s_wpart[it & 1][threadIdx.x >> 5][0] = a;
    };
    auto flushf = [&](uint32_t h, int it) {
        double a = 0.0;
        for (int w = 0; w < BLK_NT / 32; ++w) a += s_wpart[it & 1][w][0];
        part[h] = a;
    };
    if constexpr (Row::kPerBond)
        blk_sweep<float, NC, true, Row>(P, (const unsigned char *)qc, GF32{}, S->sched, pref,
                                        [&](uint32_t off, uint32_t r, float xo, float sv, float qpr) {
                                            rowu(off, r, xo, fmaf((float)P.pb_g0, xo, sv), qpr);
                                        },
                                        endf, flushf);
    else
        blk_sweep<float, NC, true, Row>(P, (const unsigned char *)qc, GF32{}, S->sched, pref,
                                        [&](uint32_t off, uint32_t r, float xo, const float *acc, const int *cnt, float qpr) {
                                            rowu(off, r, xo, blk_y_f32<NC>(P, acc, cnt, xo), qpr);
                                        },
                                        endf, flushf);
}


// ---------------------------------------------------------------------------------------
// Bond correlations (the adjoint of the couplings): out_b = g^T (s_u.s_v) x.  By Eq. E-2-1
// [(s_u.s_v) x]_i = x_i / 4 - (x_i - x_t) / 2 when the exchange of b is allowed at row i
// (x_t its target) and x_i / 4 otherwise, so out_b = T0 / 4 - C_b / 2 with T0 = g.x and
// C_b = sum over the rows where b's spins differ of g_i (x_i - x_t).  One launch serves the
// Row::kNB bonds of a chunk plan (bcmode); every thread keeps their C_b and T0 in registers
// over its rows, and part[cta][k] (k = kNB: T0) gets the CTA sums (fixed order, static block
// schedule, so the result does not depend on timing).  FP64: x is gathered as fixed point
// of exponent E (units 2^(E - 1022 - FIX_BITS)), FP32: as float.
template <class T> struct BcSv { using S = int64_t; };
template <> struct BcSv<float> { using S = float; };

// acc += g_i d for one bond: double-float arithmetic on the FP32 pipe (GB300 runs binary64
// multiply-adds and int64 -> binary64 conversions at about 1/70 of the FP32 rate); d is the
// exact fixed-point difference x_i - x_t (an integer below 2^54) or a float difference
__device__ __forceinline__ void bc_mac(ef::df &acc, const ef::df &gi, int64_t d) {
    acc = ef::df_add(acc, ef::df_mul(gi, ef::df_from_fix(d, 1022 + ef::FIX_BITS, 0, 0)));
}
__device__ __forceinline__ void bc_mac(ef::df &acc, const ef::df &gi, float d) {
    acc = ef::df_add(acc, ef::df_mulf(gi, d));
}

template <class T, class Row, class Sv, class G>
__device__ __forceinline__ void bc_sweep(const BlkParams &P, const T *__restrict__ x, const T *__restrict__ g,
                                         const G &gx, ef::df *acc, double &t0) {
    blk_sweep<Sv, 1, false, Row>(
        P, (const unsigned char *)x, gx, nullptr, [&](uint32_t i) { return (double)g[i]; },
        [&](uint32_t, uint32_t r, Sv xo, double gi, const BlkMeta &B, const unsigned char *Xsb, uint32_t l) {
            t0 = fma(gi, (double)xo, t0);
            const ef::df gd = ef::df_from_bits(ef::d2u(gi), 0);
            Row::template sums_bc<Sv>(P, B, Xsb, (const unsigned char *)x, l, r, gx, xo, gd, acc);
        },
        [](int) {}, [](uint32_t, int) {});
}

template <class T, class Row>
__device__ __forceinline__ void bc_body(const BlkParams &P, const T *__restrict__ x, const T *__restrict__ g,
                                        const int *__restrict__ Eptr, double *__restrict__ part) {
    using Sv = typename BcSv<T>::S;
    ef::df acc[Row::kNB];
#pragma unroll
    for (int k = 0; k < Row::kNB; ++k) acc[k] = ef::df{0.0f, 0.0f};
    double t0 = 0.0;
    if constexpr (sizeof(T) == 8) bc_sweep<T, Row, Sv>(P, x, g, GF64{Eptr ? *Eptr : 0}, acc, t0);
    else bc_sweep<T, Row, Sv>(P, x, g, GF32{}, acc, t0);
    __shared__ double red[BLK_NT / 32];
    double *pc = part + (size_t)blockIdx.x * (Row::kNB + 1);
#pragma unroll
    for (int k = 0; k < Row::kNB; ++k) {
        const double v = block_sum<BLK_NT>((double)acc[k].hi + (double)acc[k].lo, red);
        if (threadIdx.x == 0) pc[k] = v;
    }
    const double v = block_sum<BLK_NT>(t0, red);
    if (threadIdx.x == 0) pc[Row::kNB] = v;
}

}  // namespace hm
