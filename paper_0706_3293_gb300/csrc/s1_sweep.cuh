// s1_sweep.cuh -- plan and device bodies of the s = 1 block-structured products
// (s1blk.cu); compiles under nvcc and NVRTC alike.
//
// The rank of Sec. 3.2 is additive over positions for any spin, so with the low part l
// (sites 0..K-1, two bits per site) and the high part h (sites K..N-1) of a state
//     index = off(h) + rank_K(l),   off(h) = sum_{p >= K} CD[p][S_p][a_p],
// where the running digit sums S_p of the high positions start from k = A - sum(h), the
// digit sum of the low part; the states with the same h form one contiguous block of
// D(K, k) rows in rank_K order.  For s = 1 every allowed exchange element
// 1/2 s+_u s-_v is 1 (Eq. E-2-1 with the ladder factors sqrt(2) sqrt(2) / 2), so an
// exchange adds -J_b x_t; the diagonal is -J_b m_u m_v with m = 1 - a.
//
// The bodies below serve the kernels compiled at run time for one bond list (jit.cu):
// the bond terms of the low sites are written out, and every exchange target among the
// low words is read from a rank table indexed by the row's position g in the list of low
// words (coalesced reads; two 16-bit ranks per entry, the low half for direction d = 0,
// the high half for d = 1; 0xFFFF where the exchange is not allowed):
//   rl[pi nlw + g]: site pair pi = q (q - 1) / 2 + p (p < q < K), d = 0: l - e_p + e_q,
//                   d = 1: l + e_p - e_q, rank within the same digit sum;
//   rx[p nlw + g]:  d = 0: l - e_p (digit sum k - 1), d = 1: l + e_p (k + 1).
// Exchanges among the high sites read the same row of another block (one offset per
// block), exchanges across the split a row of a block one unit of digit sum away.
#pragma once

#include "hm_dev.cuh"
#include "ef64.cuh"

namespace hm {

constexpr int S1_NT = 512;
constexpr int S1_MAXB = 96;          // bonds of each kind
constexpr int S1_LWOFF = 22;         // entries of S1Plan::lwoff (>= 2 K + 2)
constexpr int S1_MAXK = 10;          // low sites at most

struct S1Plan {
    int N, K, H, A, nblocks, max_block;
    const uint16_t *lut;             // [4^K]: rank_K of each packed low word among words of its digit sum
    const uint32_t *lw;              // packed low words by digit sum k, each run in rank order
    const uint4 *blocks;             // per block, in row order: {h, off, k, rows}
    const uint32_t *cd;              // the sector's CD table (cd_w, cd_rowlen as in SectorView)
    int cd_w, cd_rowlen, cd_len;
    int lwoff[S1_LWOFF];             // digit sum k owns lw[lwoff[k] .. lwoff[k + 1])
    int nlo, nhi, ncr;
    uint8_t lo_p[S1_MAXB], lo_q[S1_MAXB];   // both ends below K
    uint8_t hi_p[S1_MAXB], hi_q[S1_MAXB];   // both ends at K or above (relative to K)
    uint8_t cr_p[S1_MAXB], cr_q[S1_MAXB];   // low end p, high end q (relative to K)
    float lo_j[S1_MAXB], hi_j[S1_MAXB], cr_j[S1_MAXB];   // -J_b
    // exchange rank tables of the low words (see above; independent of the couplings)
    int nlw;                         // low words in the lists: lwoff[2K + 1]
    const uint32_t *rl, *rx;
    // FP64: the couplings as integers C_b = round(-J_b 2^cs), |C_b| <= 2^52
    int cs;
    long long lo_c[S1_MAXB], hi_c[S1_MAXB], cr_c[S1_MAXB];
};

__device__ __forceinline__ int s1_dig(uint32_t w, int p) { return (int)((w >> (2 * p)) & 3u); }

// off(h) for a block whose low part has digit sum k (cd: the CD table in shared memory)
__device__ __forceinline__ uint32_t s1_off(const S1Plan &P, const uint32_t *cd, uint32_t h, int k) {
    int S = k;
    uint32_t off = 0;
    for (int t = 0; t < P.H; ++t) {
        const int a = s1_dig(h, t);
        S += a;
        off += cd[(P.K + t) * P.cd_rowlen + S * P.cd_w + a];
    }
    return off;
}

// ---- per-block set-up of the specialised bodies -------------------------------------------
// Cf: coupling type (float -J_b in FP32, integer C_b in FP64)
template <class Cf> struct S1Hi {  // a valid high exchange: target block offset, coupling
    uint32_t t;
    Cf c;
};
template <class Cf> struct S1Blk {
    uint32_t raw[2 * S1_MAXB];       // high exchange (bond, direction): target block or ~0
    S1Hi<Cf> hx[2 * S1_MAXB];        // the valid ones, compacted in bond order
    uint32_t cb[2 * S1_MAXB];        // cross exchange (bond, direction): target block or ~0
    int8_t cm[S1_MAXB];              // cross bond: m of its high site in this block
    Cf cc[S1_MAXK];                  // low site p: sum over its cross bonds of coupling x m_q
    Cf bdiag;                        // diagonal of the high bonds
    int nh;
};

template <class Cf> __device__ __forceinline__ Cf s1_cpl_hi(const S1Plan &P, int j);
template <> __device__ __forceinline__ float s1_cpl_hi<float>(const S1Plan &P, int j) { return P.hi_j[j]; }
template <> __device__ __forceinline__ long long s1_cpl_hi<long long>(const S1Plan &P, int j) { return P.hi_c[j]; }
template <class Cf> __device__ __forceinline__ Cf s1_cpl_cr(const S1Plan &P, int j);
template <> __device__ __forceinline__ float s1_cpl_cr<float>(const S1Plan &P, int j) { return P.cr_j[j]; }
template <> __device__ __forceinline__ long long s1_cpl_cr<long long>(const S1Plan &P, int j) { return P.cr_c[j]; }

// phase 1 (before a barrier): neighbouring blocks of the high and cross exchanges, the
// high-site diagonal
template <class Cf>
__device__ __forceinline__ void s1_setup(const S1Plan &P, const uint32_t *cd, uint32_t h, int k, S1Blk<Cf> &sb) {
    const int tid = threadIdx.x;
    if (tid < 2 * P.nhi) {
        const int j = tid >> 1, d = tid & 1, p = P.hi_p[j], q = P.hi_q[j];
        const int ap = s1_dig(h, p), aq = s1_dig(h, q);
        const bool ok = d == 0 ? (ap >= 1 && aq <= 1) : (ap <= 1 && aq >= 1);
        const uint32_t h2 = d == 0 ? h - (1u << (2 * p)) + (1u << (2 * q)) : h + (1u << (2 * p)) - (1u << (2 * q));
        sb.raw[tid] = ok ? s1_off(P, cd, h2, k) : 0xFFFFFFFFu;
    } else if (tid >= 256 && tid < 256 + 2 * P.ncr) {
        const int e = tid - 256, j = e >> 1, d = e & 1, q = P.cr_q[j];
        const int aq = s1_dig(h, q);
        // d = 0: the low site gives a unit to the high site (k - 1); d = 1: the reverse
        const int k2 = d == 0 ? k - 1 : k + 1;
        const bool ok = (d == 0 ? aq <= 1 : aq >= 1) && k2 >= 0 && k2 <= 2 * P.K;
        const uint32_t h2 = d == 0 ? h + (1u << (2 * q)) : h - (1u << (2 * q));
        sb.cb[e] = ok ? s1_off(P, cd, h2, k2) : 0xFFFFFFFFu;
        if (d == 0) sb.cm[j] = (int8_t)(1 - aq);
    }
    if (tid == S1_NT - 1) {
        Cf dsum = 0;
        for (int j = 0; j < P.nhi; ++j)
            dsum += s1_cpl_hi<Cf>(P, j) * (Cf)((1 - s1_dig(h, P.hi_p[j])) * (1 - s1_dig(h, P.hi_q[j])));
        sb.bdiag = dsum;
    }
}

// phase 2 (between two barriers): warp 0 compacts the valid high exchanges (ballots, bond
// order kept), warp 1 sums the cross couplings of each low site
template <class Cf>
__device__ __forceinline__ void s1_compact(const S1Plan &P, S1Blk<Cf> &sb) {
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    if (warp == 0) {
        int base = 0;
        for (int c = 0; c < 2 * P.nhi; c += 32) {
            const int e = c + lane;
            const uint32_t t = e < 2 * P.nhi ? sb.raw[e] : 0xFFFFFFFFu;
            const bool v = t != 0xFFFFFFFFu;
            const uint32_t b = __ballot_sync(0xffffffffu, v);
            if (v) {
                const int o = base + __popc(b & ((1u << lane) - 1u));
                sb.hx[o].t = t;
                sb.hx[o].c = s1_cpl_hi<Cf>(P, e >> 1);
            }
            base += __popc(b);
        }
        if (lane == 0) sb.nh = base;
    } else if (warp == 1 && lane < P.K) {
        Cf c = 0;
        for (int j = 0; j < P.ncr; ++j)
            if (P.cr_p[j] == lane) c += s1_cpl_cr<Cf>(P, j) * (Cf)sb.cm[j];
        sb.cc[lane] = c;
    }
}

// ---- FP32: y = H x (LZ false) or the Lanczos product u = sigma H q - gamma q_prev over
// q_prev with part[block] = (sigma q . u) (LZ true) -------------------------------------------
template <class Row, bool LZ>
__device__ __forceinline__ void s1j_body32(const S1Plan &P, const float *__restrict__ x, float *__restrict__ y,
                                           const LzScalars *__restrict__ S, double *__restrict__ part) {
    if constexpr (LZ) {
        if (S->done) return;
    }
    extern __shared__ __align__(16) unsigned char smem[];
    uint32_t *cd = (uint32_t *)smem;                                   // [cd_len]
    float *Xs = (float *)(smem + ((P.cd_len * 4 + 15) & ~15));         // [max_block]
    __shared__ S1Blk<float> sb;
    __shared__ double red[S1_NT / 32];
    const int tid = threadIdx.x;
    for (int i = tid; i < P.cd_len; i += S1_NT) cd[i] = P.cd[i];
    float sg = 1.0f, gm = 0.0f;
    if constexpr (LZ) {
        sg = (float)S->sigma_cur;
        gm = (float)(S->beta_prev * S->sigma_prev);
    }
    __syncthreads();
    for (int bi = blockIdx.x; bi < P.nblocks; bi += gridDim.x) {
        const uint4 bk = P.blocks[bi];
        const uint32_t h = bk.x, off = bk.y;
        const int k = (int)bk.z, n = (int)bk.w;
        s1_setup<float>(P, cd, h, k, sb);
        for (int r = tid; r < n; r += S1_NT) Xs[r] = x[off + r];
        __syncthreads();
        s1_compact<float>(P, sb);
        __syncthreads();
        const uint32_t lwb = (uint32_t)P.lwoff[k];
        const int nh = sb.nh;
        ef::df dot{0.0f, 0.0f};
        for (int r = tid; r < n; r += S1_NT) {
            const uint32_t g = lwb + (uint32_t)r;
            const uint32_t l = __ldg(P.lw + g);
            const float xo = Xs[r];
            float dg = sb.bdiag, acc = 0.0f;
            Row::row32(l, Xs, x, P.rl + g, P.rx + g, sb.cb, sb.cc, dg, acc);
            // four high gathers a round, the last round's loads past the list predicated off
            // (no serial tail); the multiply-adds keep the list order
            for (int e = 0; e < nh; e += 4) {
                float cv[4], xv[4];
#pragma unroll
                for (int i = 0; i < 4; ++i) {
                    if (e + i < nh) {
                        const S1Hi<float> he = sb.hx[e + i];
                        cv[i] = he.c;
                        xv[i] = __ldg(x + (he.t + (uint32_t)r));
                    } else {
                        cv[i] = 0.0f;
                        xv[i] = 0.0f;
                    }
                }
#pragma unroll
                for (int i = 0; i < 4; ++i) acc = fmaf(cv[i], xv[i], acc);
            }
            const float hv = fmaf(dg, xo, acc);
            if constexpr (LZ) {
                const float u = sg * hv - gm * y[off + r];
                y[off + r] = u;
                dot = ef::df_add(dot, ef::two_prod(sg * xo, u));
            } else {
                y[off + r] = hv;
            }
        }
        if constexpr (LZ) {
            const double t = block_sum<S1_NT>((double)dot.hi + (double)dot.lo, red);
            if (tid == 0) part[bi] = t;
        }
        __syncthreads();                 // the next block's set-up overwrites this one's
    }
}

// value of a 128-bit integer (|T| < 2^117) as a double: the high word exactly, the low
// word and the sum rounded (within one unit in the last place)
__device__ __forceinline__ double s1_i128_to_double(__int128 v) {
    const long long hi = (long long)(v >> 64);
    const unsigned long long lo = (unsigned long long)v;
    return (double)hi * 18446744073709551616.0 + (double)lo;
}

// ---- FP64 Lanczos product: Xc = q_cur as fixed point of exponent E = S->emax[pc] (unit
// 2^u, u = E - 1022 - FIX_BITS, |X| <= 2^53 + 1); every row is one exact int128 sum
//     T = (sum_b C_b m_u m_v) X_i + sum_b C_b (sum over b's allowed exchanges of X_t)
// (|C_b| <= 2^52, so |T| < 2^116 for up to 288 bonds), converted to binary64 and scaled,
// y_i = T 2^(u - cs), into Y (bit patterns); part[block] = (q . y) over the block's rows
// (double-float products and sums: no binary64 instruction per row for the dot).
template <class Row>
__device__ __forceinline__ void s1j_body64(const S1Plan &P, const long long *__restrict__ Xc,
                                           unsigned long long *__restrict__ Y, const LzScalars *__restrict__ S, int pc,
                                           double *__restrict__ part) {
    if (S->done) return;
    const int E = S->emax[pc];
    const int u = E - 1022 - ef::FIX_BITS;
    const double sy = ef::pow2d(u - P.cs);
    extern __shared__ __align__(16) unsigned char smem[];
    uint32_t *cd = (uint32_t *)smem;                                        // [cd_len]
    long long *Xs = (long long *)(smem + ((P.cd_len * 4 + 15) & ~15));      // [max_block]
    __shared__ S1Blk<long long> sb;
    __shared__ double red[S1_NT / 32];
    const int tid = threadIdx.x;
    for (int i = tid; i < P.cd_len; i += S1_NT) cd[i] = P.cd[i];
    __syncthreads();
    for (int bi = blockIdx.x; bi < P.nblocks; bi += gridDim.x) {
        const uint4 bk = P.blocks[bi];
        const uint32_t h = bk.x, off = bk.y;
        const int k = (int)bk.z, n = (int)bk.w;
        s1_setup<long long>(P, cd, h, k, sb);
        for (int r = tid; r < n; r += S1_NT) Xs[r] = Xc[off + r];
        __syncthreads();
        s1_compact<long long>(P, sb);
        __syncthreads();
        const uint32_t lwb = (uint32_t)P.lwoff[k];
        const int nh = sb.nh;
        ef::df d1f{0.0f, 0.0f};
        for (int r = tid; r < n; r += S1_NT) {
            const uint32_t g = lwb + (uint32_t)r;
            const uint32_t l = __ldg(P.lw + g);
            const long long xo = Xs[r];
            long long dg = sb.bdiag;
            __int128 a = 0;
            Row::row64(l, Xs, Xc, P.rl + g, P.rx + g, sb.cb, sb.cc, dg, a);
            // two high gathers a round, the last round's second load predicated off
            for (int e = 0; e < nh; e += 2) {
                long long cv[2], xv[2];
#pragma unroll
                for (int i = 0; i < 2; ++i) {
                    if (e + i < nh) {
                        const S1Hi<long long> he = sb.hx[e + i];
                        cv[i] = he.c;
                        xv[i] = __ldg(Xc + (he.t + (uint32_t)r));
                    } else {
                        cv[i] = 0;
                        xv[i] = 0;
                    }
                }
#pragma unroll
                for (int i = 0; i < 2; ++i) a += (__int128)xv[i] * cv[i];
            }
            const __int128 t = a + (__int128)dg * xo;
            const unsigned long long yb = ef::d2u(s1_i128_to_double(t) * sy);
            __stcs(Y + off + r, yb);
            d1f = ef::df_add(d1f, ef::df_mul(ef::df_from_fix(xo, E, 0, E - 1023), ef::df_from_bits(yb, E - 1023)));
        }
        const double q_y = ldexp((double)d1f.hi + (double)d1f.lo, 2 * (E - 1023));
        const double tsum = block_sum<S1_NT>(q_y, red);
        if (tid == 0) part[bi] = tsum;
        __syncthreads();
    }
}

}  // namespace hm
