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

// Per-thread scratch of the prefix form of the target encode (row_apply, PX = true):
// prefix sums P+[r], P-[r] of the rank-term changes a +-1 shift of the running digit sum
// causes at positions 1..r, and the running digit sums S[r].  Laid out [slot][thread]:
// the threads of a warp visit the same bond together, so they read the same slot of
// consecutive threads (no bank conflict).
constexpr int ROW_NT = 256;          // threads per CTA of the row kernels
template <class I>
__host__ __device__ __forceinline__ size_t row_px_bytes(const SectorView &sv) {
    const size_t a = (size_t)2 * sv.N * ROW_NT * sizeof(I);
    return ((a + 15) & ~(size_t)15) + (((size_t)sv.N * ROW_NT + 15) & ~(size_t)15);
}
// the prefix form is used while its scratch stays below this (else the per-hop walk)
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
// per-thread scratch of row_px_bytes) the row first forms the prefix sums of those
// changes, P_dp[r] = sum_{t=1..r} (CD[t][S_t + dp][a_t] - CD[t][S_t][a_t]), so that every
// exchange costs its two end terms and P_dp[q-1] - P_dp[p]; without it each exchange
// walks positions p..q (Codec::delta).
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
    const int N = c.N, nt = ROW_NT;
    I *Pp = px, *Pm = px + (size_t)N * nt;
    uint8_t *Ss = px ? reinterpret_cast<uint8_t *>(px - threadIdx.x) + (((size_t)2 * N * nt * sizeof(I) + 15) & ~(size_t)15) +
                           threadIdx.x
                     : nullptr;
    if (px) {
        int S = dig(w, 0, bits);
        I pp = 0, pm = 0;
        Pp[0] = 0;
        Pm[0] = 0;
        Ss[0] = (uint8_t)S;
        for (int r = 1; r < N; ++r) {
            const int a = dig(w, r, bits);
            S += a;
            const I t0 = c.at(r, S, a);
            pp += (S < c.A ? c.at(r, S + 1, a) : t0) - t0;
            pm += (S > 0 ? c.at(r, S - 1, a) : t0) - t0;
            Pp[(size_t)r * nt] = pp;
            Pm[(size_t)r * nt] = pm;
            Ss[(size_t)r * nt] = (uint8_t)S;
        }
    }
    // index change of the exchange (p, q, dp) from the prefix sums
    auto delta_px = [&](int p, int q, int ap, int aq, int dp) -> I {
        const int Sq = Ss[(size_t)q * nt];
        const I *P = dp > 0 ? Pp : Pm;
        I d = P[(size_t)(q - 1) * nt] - P[(size_t)p * nt] + (c.at(q, Sq, aq - dp) - c.at(q, Sq, aq));
        if (p >= 1) {
            const int Sp = Ss[(size_t)p * nt];
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
