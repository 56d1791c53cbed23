// hm_row.cuh -- the per-row kernel body of Eq. (E-4-b): apply every bond term of
// Eq. (E-2-1) to the row's own basis state, encode each target, gather x there.
#pragma once

#include "hm_internal.cuh"

namespace hm {

// Tables one CTA needs in shared memory: the exchange factors, then the rank table CD.
// Layout: double hs[128] | float hsf[128] | CD.  hs[0..64) = pdn, hs[64..128) = pup.
template <class I>
__device__ __forceinline__ I *stage_tables(const SectorView &sv, const BondParams &bp,
                                           unsigned char *smem_raw, const double **pdn,
                                           const double **pup) {
    double *hs = reinterpret_cast<double *>(smem_raw);
    float *hsf = reinterpret_cast<float *>(smem_raw + 128 * sizeof(double));
    I *cd = reinterpret_cast<I *>(smem_raw + 128 * sizeof(double) + 128 * sizeof(float));
    for (int k = threadIdx.x; k < 64; k += blockDim.x) {
        hs[k] = bp.hs_pdn[k];
        hs[64 + k] = bp.hs_pup[k];
        hsf[k] = (float)bp.hs_pdn[k];
        hsf[64 + k] = (float)bp.hs_pup[k];
    }
    for (int k = threadIdx.x; k < sv.cd_len; k += blockDim.x) cd[k] = ((const I *)sv.cd)[k];
    __syncthreads();
    *pdn = hs;
    *pup = hs + 64;
    return cd;
}

// Per-thread scratch of the suffix form of the target encode (row_apply with px): suffix
// sums Q+[r], Q-[r] (r = 1..N, Q[N] = 0) of the rank-term changes a +-1 shift of the
// running digit sum causes at positions r..N-1, and the running digit sums S[r].  Laid
// out [slot][thread]: the threads of a warp visit the same bond together, so they read
// the same slot of consecutive threads (no bank conflict).
constexpr int ROW_NT = 256;          // threads per CTA of the row kernels
template <class I>
__host__ __device__ __forceinline__ size_t row_px_bytes(const SectorView &sv) {
    const size_t a = (size_t)2 * (sv.N + 1) * ROW_NT * sizeof(I);
    return ((a + 15) & ~(size_t)15) + (((size_t)sv.N * ROW_NT + 15) & ~(size_t)15);
}
// the suffix form is used while its scratch stays below this (else the per-hop walk)
constexpr size_t ROW_PX_MAX = 96 * 1024;

template <class I>
__host__ __forceinline__ size_t row_smem_bytes(const SectorView &sv) {
    size_t b = 128 * sizeof(double) + 128 * sizeof(float) + (size_t)sv.cd_len * sizeof(I);
    b = (b + 15) & ~(size_t)15;
    if (row_px_bytes<I>(sv) <= ROW_PX_MAX) b += row_px_bytes<I>(sv);
    return b;
}

// scratch of the prefix form for this thread (nullptr when the walk is used)
template <class I>
__device__ __forceinline__ I *row_px_base(const SectorView &sv, unsigned char *smem_raw) {
    if (row_px_bytes<I>(sv) > ROW_PX_MAX) return nullptr;
    size_t b = 128 * sizeof(double) + 128 * sizeof(float) + (size_t)sv.cd_len * sizeof(I);
    b = (b + 15) & ~(size_t)15;
    return reinterpret_cast<I *>(smem_raw + b) + threadIdx.x;
}

// views of the per-thread scratch (px = row_px_base; nullptr = no scratch)
template <class I>
struct RowPx {
    I *Qp, *Qm;          // [r * ROW_NT], r = 0..N
    uint8_t *S;          // [r * ROW_NT], r = 0..N-1
    __device__ __forceinline__ RowPx(I *px, int N) {
        Qp = px;
        Qm = px ? px + (size_t)(N + 1) * ROW_NT : nullptr;
        S = px ? reinterpret_cast<uint8_t *>(px - threadIdx.x) +
                     (((size_t)2 * (N + 1) * ROW_NT * sizeof(I) + 15) & ~(size_t)15) + threadIdx.x
               : nullptr;
    }
};

// running digit sums and suffix sums of the rank-term changes of positions lo..hi (descending
// from hi, whose running sum S_hi is given; Q[hi + 1] must be current)
template <class I>
__device__ __forceinline__ void px_fill(const Codec<I> &c, uint64_t w, const RowPx<I> &x, int hi, int S) {
    I qp = x.Qp[(size_t)(hi + 1) * ROW_NT], qm = x.Qm[(size_t)(hi + 1) * ROW_NT];
    for (int r = hi; r >= 0; --r) {
        const int a = dig(w, r, c.bits);
        x.S[(size_t)r * ROW_NT] = (uint8_t)S;
        if (r >= 1) {
            const I t0 = c.at(r, S, a);
            qp += (S < c.A ? c.at(r, S + 1, a) : t0) - t0;
            qm += (S > 0 ? c.at(r, S - 1, a) : t0) - t0;
            x.Qp[(size_t)r * ROW_NT] = qp;
            x.Qm[(size_t)r * ROW_NT] = qm;
        }
        S -= a;
    }
}

// scratch for state w (all positions)
template <class I>
__device__ __forceinline__ void px_full(const Codec<I> &c, uint64_t w, const RowPx<I> &x) {
    x.Qp[(size_t)c.N * ROW_NT] = 0;
    x.Qm[(size_t)c.N * ROW_NT] = 0;
    px_fill(c, w, x, c.N - 1, c.A);
}

// Successor rule (Sec. 3.1): the state of the next index.  The lowest position k whose
// digit can give one unit to position k+1 does so, and the units left at positions
// 0..k are refilled from the bottom, at most 2s each.  Returns k (digits 0..k+1 changed;
// the running digit sums above are unchanged), or -1 for the last state of the sector.
__device__ __forceinline__ int successor_word(uint64_t &w, int N, int S2, int bits) {
    const uint64_t m = (1ull << bits) - 1ull;
    int units = 0, k = -1;
    for (int p = 0; p + 1 < N; ++p) {
        const int a = (int)((w >> (p * bits)) & m);
        units += a;
        if (a > 0 && (int)((w >> ((p + 1) * bits)) & m) < S2) { k = p; break; }
    }
    if (k < 0) return -1;
    w += 1ull << ((k + 1) * bits);
    w &= ~((1ull << ((k + 1) * bits)) - 1ull);
    units -= 1;
    for (int p = 0; p <= k && units > 0; ++p) {
        const int t = units < S2 ? units : S2;
        w |= (uint64_t)t << (p * bits);
        units -= t;
    }
    return k;
}

// every row of this thread's share.  run = 1: one row per thread per grid stride, each
// decoded (Sec. 3.1 decode rule; consecutive threads take consecutive rows, so the row
// loads coalesce).  run > 1: runs of `run` consecutive rows per thread, the first decoded
// and the others reached by the successor rule, the scratch (if any) following the state
// incrementally.  f(row, w) sees the scratch of w.
template <class I, class F>
__device__ __forceinline__ void row_runs(const Codec<I> &c, uint64_t dim, I *px, int run, F &&f) {
    const RowPx<I> x(px, c.N);
    const uint64_t stride = (uint64_t)gridDim.x * blockDim.x;
    if (run <= 1) {
        for (uint64_t r = blockIdx.x * (uint64_t)blockDim.x + threadIdx.x; r < dim; r += stride) {
            const uint64_t w = c.decode((I)r);
            if (px) px_full(c, w, x);
            f(r, w);
        }
        return;
    }
    const uint64_t nruns = (dim + run - 1) / run;
    for (uint64_t k0 = blockIdx.x * (uint64_t)blockDim.x + threadIdx.x; k0 < nruns; k0 += stride) {
        uint64_t r = k0 * run;
        const uint64_t rend = r + run < dim ? r + run : dim;
        uint64_t w = c.decode((I)r);
        if (px) px_full(c, w, x);
        for (;;) {
            f(r, w);
            if (++r >= rend) break;
            const int k = successor_word(w, c.N, c.S2, c.bits);
            if (px) px_fill(c, w, x, k + 1, x.S[(size_t)(k + 1) * ROW_NT]);
        }
    }
}

// run length of the row kernels: HM_ROW_RUN (1..64, default 1)
int row_run_len();

template <class Acc>
__device__ __forceinline__ Acc jm_of(const BondParams &bp, int t) {
    if constexpr (sizeof(Acc) == 8) return (Acc)bp.jm[t];
    else return (Acc)bp.jmf[t];
}

// (H x)_i for NV vector columns of a row-major [dim][ld] array starting at column c0.
// T is the storage type, Acc the accumulation type.  Returns the diagonal element in
// *diag_out (as Acc) and the off-diagonal sum in acc[]; the caller forms
// y = diag * x_i + acc, the same association as the oracle's row.
//
// Target encode (Sec. 3.2): an exchange moves the digit at p by dp and the one at q > p by
// -dp, so only the rank terms of positions p..q change, and those strictly between p and
// q change only through their running digit sum (S_r -> S_r + dp).  With px (the
// per-thread scratch of row_px_bytes, describing w: px_full / row_runs) every exchange
// costs its two end terms and Q_dp[p+1] - Q_dp[q], the suffix sums
// Q_dp[r] = sum_{t=r..N-1} (CD[t][S_t + dp][a_t] - CD[t][S_t][a_t]); without it each
// exchange walks positions p..q (Codec::delta).
template <class I, class T, class Acc, int NV>
__device__ __forceinline__ void row_apply(const Codec<I> &c, const BondParams &bp,
                                          const double *hs_pdn, const double *hs_pup,
                                          I i, uint64_t w, const T *__restrict__ x, int ld,
                                          int c0, Acc *acc, Acc *diag_out, I *px = nullptr) {
    const int S2 = c.S2, bits = c.bits;
    // coefficients in the accumulation type: an FP32 product never touches the FP64 pipe
    const Acc half = Acc(0.5) * Acc(S2);
    // pdn table base; pup = pdn + 64 (doubles) -- for floats the copy starts 128 doubles in
    const Acc *tpdn, *tpup;
    if constexpr (sizeof(Acc) == 8) {
        tpdn = reinterpret_cast<const Acc *>(hs_pdn);
        tpup = reinterpret_cast<const Acc *>(hs_pup);
    } else {
        tpdn = reinterpret_cast<const Acc *>(hs_pdn + 128);
        tpup = tpdn + 64;
    }
    Acc dg = Acc(0);
#pragma unroll
    for (int k = 0; k < NV; ++k) acc[k] = Acc(0);
    const RowPx<I> sx(px, c.N);
    // index change of the exchange (p, q, dp) from the suffix sums of the scratch
    auto delta_px = [&](int p, int q, int ap, int aq, int dp) -> I {
        const int Sq = sx.S[(size_t)q * ROW_NT];
        const I *Q = dp > 0 ? sx.Qp : sx.Qm;
        I d = Q[(size_t)(p + 1) * ROW_NT] - Q[(size_t)q * ROW_NT] + (c.at(q, Sq, aq - dp) - c.at(q, Sq, aq));
        if (p >= 1) {
            const int Sp = sx.S[(size_t)p * ROW_NT];
            d += c.at(p, Sp + dp, ap + dp) - c.at(p, Sp, ap);
        }
        return d;
    };
    for (int t = 0; t < bp.nb; ++t) {
        const int p = bp.p[t], q = bp.q[t];
        const int ap = dig(w, p, bits), aq = dig(w, q, bits);
        const Acc jm = jm_of<Acc>(bp, t);
        dg += jm * (half - Acc(ap)) * (half - Acc(aq));
        if (ap >= 1 && aq < S2) {          // s+_p s-_q
            const I j = i + (px ? delta_px(p, q, ap, aq, -1) : c.delta(w, p, q, -1));
            const Acc cf = jm * tpdn[ap * 8 + aq];
            const T *xr = x + (size_t)j * ld + c0;
#pragma unroll
            for (int k = 0; k < NV; ++k) acc[k] += cf * (Acc)xr[k];
        }
        if (ap < S2 && aq >= 1) {          // s-_p s+_q
            const I j = i + (px ? delta_px(p, q, ap, aq, +1) : c.delta(w, p, q, +1));
            const Acc cf = jm * tpup[ap * 8 + aq];
            const T *xr = x + (size_t)j * ld + c0;
#pragma unroll
            for (int k = 0; k < NV; ++k) acc[k] += cf * (Acc)xr[k];
        }
    }
    *diag_out = dg;
}

}  // namespace hm
