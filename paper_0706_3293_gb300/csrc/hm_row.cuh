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

template <class I>
__host__ __forceinline__ size_t row_smem_bytes(const SectorView &sv) {
    return 128 * sizeof(double) + 128 * sizeof(float) + (size_t)sv.cd_len * sizeof(I);
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
template <class I, class T, class Acc, int NV>
__device__ __forceinline__ void row_apply(const Codec<I> &c, const BondParams &bp,
                                          const double *hs_pdn, const double *hs_pup,
                                          I i, uint64_t w, const T *__restrict__ x, int ld,
                                          int c0, Acc *acc, Acc *diag_out) {
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
    for (int t = 0; t < bp.nb; ++t) {
        const int p = bp.p[t], q = bp.q[t];
        const int ap = dig(w, p, bits), aq = dig(w, q, bits);
        const Acc jm = jm_of<Acc>(bp, t);
        dg += jm * (half - Acc(ap)) * (half - Acc(aq));
        if (ap >= 1 && aq < S2) {          // s+_p s-_q
            const I j = i + c.delta(w, p, q, -1);
            const Acc cf = jm * tpdn[ap * 8 + aq];
            const T *xr = x + (size_t)j * ld + c0;
#pragma unroll
            for (int k = 0; k < NV; ++k) acc[k] += cf * (Acc)xr[k];
        }
        if (ap < S2 && aq >= 1) {          // s-_p s+_q
            const I j = i + c.delta(w, p, q, +1);
            const Acc cf = jm * tpup[ap * 8 + aq];
            const T *xr = x + (size_t)j * ld + c0;
#pragma unroll
            for (int k = 0; k < NV; ++k) acc[k] += cf * (Acc)xr[k];
        }
    }
    *diag_out = dg;
}

}  // namespace hm
