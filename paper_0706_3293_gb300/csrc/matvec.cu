// matvec.cu -- y = H x by rows (Eq. E-4-b), the bond-correlation adjoint, start vectors.
#include "hm_row.cuh"

namespace hm {

// ---------------------------------------------------------------------------------------
// general row kernel: one thread per output row, grid-stride over rows
// ---------------------------------------------------------------------------------------
template <class I, class T, class Acc, int NV>
__global__ void __launch_bounds__(256)
k_matvec(SectorView sv, BondParams bp, const T *__restrict__ x, T *__restrict__ y, int ld, int c0) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    const double *pdn, *pup;
    const I *cd = stage_tables<I>(sv, bp, smem_raw, &pdn, &pup);
    Codec<I> c{cd, sv.N, sv.S2, sv.A, sv.bits, sv.cd_w, sv.cd_rowlen};
    const uint64_t stride = (uint64_t)gridDim.x * blockDim.x;
    for (uint64_t r = blockIdx.x * (uint64_t)blockDim.x + threadIdx.x; r < sv.dim; r += stride) {
        const I i = (I)r;
        const uint64_t w = c.decode(i);
        Acc acc[NV], dg;
        row_apply<I, T, Acc, NV>(c, bp, pdn, pup, i, w, x, ld, c0, acc, &dg);
        const T *xi = x + r * ld + c0;
        T *yi = y + r * ld + c0;
#pragma unroll
        for (int k = 0; k < NV; ++k) yi[k] = (T)(dg * (Acc)xi[k] + acc[k]);
    }
}

template <class I, class T, class Acc, int NV>
static int launch_matvec(const SectorView &sv, const BondParams &bp, const T *x, T *y, int ld,
                         int c0, cudaStream_t st) {
    size_t sm = row_smem_bytes<I>(sv);
    HM_CUDA(cudaFuncSetAttribute(k_matvec<I, T, Acc, NV>,
                                 cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm));
    k_matvec<I, T, Acc, NV><<<grid_blocks(sv.dim, 256), 256, sm, st>>>(sv, bp, x, y, ld, c0);
    HM_CUDA(cudaGetLastError());
    return HM_OK;
}

template <class I, class T, class Acc>
static int matvec_cols(const SectorView &sv, const BondParams &bp, const T *x, T *y, int nvec,
                       cudaStream_t st) {
    int c0 = 0;
    while (c0 < nvec) {
        int rem = nvec - c0;
        int w = rem >= 32 ? 32 : rem >= 16 ? 16 : rem >= 8 ? 8 : rem >= 4 ? 4 : rem >= 2 ? 2 : 1;
        switch (w) {
            case 32: HM_TRY((launch_matvec<I, T, Acc, 32>(sv, bp, x, y, nvec, c0, st))); break;
            case 16: HM_TRY((launch_matvec<I, T, Acc, 16>(sv, bp, x, y, nvec, c0, st))); break;
            case 8: HM_TRY((launch_matvec<I, T, Acc, 8>(sv, bp, x, y, nvec, c0, st))); break;
            case 4: HM_TRY((launch_matvec<I, T, Acc, 4>(sv, bp, x, y, nvec, c0, st))); break;
            case 2: HM_TRY((launch_matvec<I, T, Acc, 2>(sv, bp, x, y, nvec, c0, st))); break;
            default: HM_TRY((launch_matvec<I, T, Acc, 1>(sv, bp, x, y, nvec, c0, st))); break;
        }
        c0 += w;
    }
    return HM_OK;
}

// ---------------------------------------------------------------------------------------
// bond correlations: out[b] = sum_i g_i [(s_u.s_v) x]_i, BC bonds per grid row
// ---------------------------------------------------------------------------------------
constexpr int BC = 16;

template <class I, class T>
__global__ void __launch_bounds__(256)
k_bond_corr(SectorView sv, BondParams bp, const T *__restrict__ g, const T *__restrict__ x,
            double *__restrict__ part) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    __shared__ double red[8];
    const double *pdn, *pup;
    const I *cd = stage_tables<I>(sv, bp, smem_raw, &pdn, &pup);
    Codec<I> c{cd, sv.N, sv.S2, sv.A, sv.bits, sv.cd_w, sv.cd_rowlen};
    const int b0 = blockIdx.y * BC;
    const int nbc = min(BC, bp.nb - b0);
    const int S2 = sv.S2, bits = sv.bits;
    const double half = 0.5 * S2;
    double acc[BC];
#pragma unroll
    for (int k = 0; k < BC; ++k) acc[k] = 0.0;
    const uint64_t stride = (uint64_t)gridDim.x * blockDim.x;
    for (uint64_t r = blockIdx.x * (uint64_t)blockDim.x + threadIdx.x; r < sv.dim; r += stride) {
        const I i = (I)r;
        const uint64_t w = c.decode(i);
        const double gi = (double)g[r], xi = (double)x[r];
#pragma unroll
        for (int k = 0; k < BC; ++k) {
            if (k < nbc) {
                const int t = b0 + k;
                const int p = bp.p[t], q = bp.q[t];
                const int ap = dig(w, p, bits), aq = dig(w, q, bits);
                double rv = (half - ap) * (half - aq) * xi;
                if (ap >= 1 && aq < S2)
                    rv += pdn[ap * 8 + aq] * (double)x[i + c.delta(w, p, q, -1)];
                if (ap < S2 && aq >= 1)
                    rv += pup[ap * 8 + aq] * (double)x[i + c.delta(w, p, q, +1)];
                acc[k] += gi * rv;
            }
        }
    }
    for (int k = 0; k < BC; ++k) {
        double s = block_sum<256>(acc[k], red);
        if (threadIdx.x == 0 && k < nbc) part[(size_t)(b0 + k) * gridDim.x + blockIdx.x] = s;
    }
}

// out[b] = sign * scale * sum_k part[b][k], k in fixed order
__global__ void k_reduce_rows(const double *__restrict__ part, int nblk, int nb, double sign,
                              const double *__restrict__ scale_div, double *__restrict__ out) {
    __shared__ double red[8];
    for (int b = blockIdx.x; b < nb; b += gridDim.x) {
        double s = 0.0;
        for (int k = threadIdx.x; k < nblk; k += blockDim.x) s += part[(size_t)b * nblk + k];
        s = block_sum<256>(s, red);
        if (threadIdx.x == 0) out[b] = sign * (scale_div ? s / *scale_div : s);
    }
}

template <class I, class T>
static int bond_corr_t(const SectorView &sv, const BondParams &bp, const T *g, const T *x,
                       double *out, double *part, int nblk, double sign, const double *div,
                       cudaStream_t st) {
    size_t sm = row_smem_bytes<I>(sv);
    HM_CUDA(cudaFuncSetAttribute(k_bond_corr<I, T>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                 (int)sm));
    dim3 grid(nblk, (bp.nb + BC - 1) / BC);
    k_bond_corr<I, T><<<grid, 256, sm, st>>>(sv, bp, g, x, part);
    HM_CUDA(cudaGetLastError());
    k_reduce_rows<<<bp.nb < 1024 ? bp.nb : 1024, 256, 0, st>>>(part, nblk, bp.nb, sign, div, out);
    HM_CUDA(cudaGetLastError());
    return HM_OK;
}

int bond_corr_dev(const hm_basis *b, const BondParams &bp, const void *g, const void *x,
                  double *out, int dtype, void *work, size_t work_bytes, double sign,
                  const double *div, cudaStream_t st) {
    const SectorView &sv = b->view;
    const int nblk = grid_blocks(sv.dim, 256);
    if (bp.nb == 0) return HM_OK;
    if (!work || work_bytes < (size_t)nblk * bp.nb * sizeof(double))
        return fail(HM_EWORKSPACE, "bond_corr needs %zu workspace bytes",
                    (size_t)nblk * bp.nb * sizeof(double));
    double *part = (double *)work;
    if (dtype == HM_F64) {
        if (sv.idx64) return bond_corr_t<uint64_t, double>(sv, bp, (const double *)g, (const double *)x, out, part, nblk, sign, div, st);
        return bond_corr_t<uint32_t, double>(sv, bp, (const double *)g, (const double *)x, out, part, nblk, sign, div, st);
    }
    if (sv.idx64) return bond_corr_t<uint64_t, float>(sv, bp, (const float *)g, (const float *)x, out, part, nblk, sign, div, st);
    return bond_corr_t<uint32_t, float>(sv, bp, (const float *)g, (const float *)x, out, part, nblk, sign, div, st);
}

size_t bond_corr_bytes(const hm_basis *b, int n_bonds) {
    return (size_t)grid_blocks(b->view.dim, 256) * (size_t)(n_bonds > 0 ? n_bonds : 1) * sizeof(double);
}

int blk_matvec(hm_basis *b, const BondParams &bp, const void *x, void *y, int dtype, int nvec,
               cudaStream_t st);

int matvec_dev(const hm_basis *b, const BondParams &bp, const void *x, void *y, int dtype,
               int nvec, cudaStream_t st) {
    const SectorView &sv = b->view;
    // s = 1/2 sectors with few coupling classes take the block path (blk.cu)
    const int brc = blk_matvec(const_cast<hm_basis *>(b), bp, x, y, dtype, nvec, st);
    if (brc <= 0) return brc;
    if (dtype == HM_F64) {
        if (sv.idx64) return matvec_cols<uint64_t, double, double>(sv, bp, (const double *)x, (double *)y, nvec, st);
        return matvec_cols<uint32_t, double, double>(sv, bp, (const double *)x, (double *)y, nvec, st);
    }
    if (sv.idx64) return matvec_cols<uint64_t, float, float>(sv, bp, (const float *)x, (float *)y, nvec, st);
    return matvec_cols<uint32_t, float, float>(sv, bp, (const float *)x, (float *)y, nvec, st);
}

// ---------------------------------------------------------------------------------------
// seeded start vectors
// ---------------------------------------------------------------------------------------
template <class T>
__global__ void k_start(uint64_t seed, int kind, uint64_t n, T *__restrict__ x) {
    for (uint64_t t = blockIdx.x * (uint64_t)blockDim.x + threadIdx.x; t < n;
         t += (uint64_t)gridDim.x * blockDim.x) {
        const uint64_t o = sm64(seed, t);
        double v = kind == 0 ? 2.0 * ((double)(o >> 11) * 0x1.0p-53) - 1.0 : ((o >> 63) ? -1.0 : 1.0);
        x[t] = (T)v;
    }
}

int start_vector_dev(uint64_t n, uint64_t seed, int kind, void *x, int dtype, cudaStream_t st) {
    int blocks = grid_blocks(n, 256);
    if (dtype == HM_F64) k_start<double><<<blocks, 256, 0, st>>>(seed, kind, n, (double *)x);
    else k_start<float><<<blocks, 256, 0, st>>>(seed, kind, n, (float *)x);
    HM_CUDA(cudaGetLastError());
    return HM_OK;
}

}  // namespace hm

using namespace hm;

extern "C" {

int matvec(const hm_basis *b, int n_bonds, const int32_t *u, const int32_t *v, const double *J,
           const void *x, void *y, int dtype, int nvec, void *stream) {
    if (!b) return fail(HM_EINVAL, "basis is NULL");
    if (dtype != HM_F64 && dtype != HM_F32) return fail(HM_EINVAL, "dtype must be HM_F64 or HM_F32");
    if (nvec < 1 || nvec > 64) return fail(HM_EINVAL, "nvec must be in 1..64 (got %d)", nvec);
    if (!x || !y) return fail(HM_EINVAL, "x or y is NULL");
    if (x == y) return fail(HM_EINVAL, "x and y must not overlap");
    BondParams bp;
    HM_TRY(make_bonds(b, n_bonds, u, v, J, &bp));
    return matvec_dev(b, bp, x, y, dtype, nvec, as_stream(stream));
}

int bond_corr_workspace(const hm_basis *b, int n_bonds, size_t *bytes) {
    if (!b || !bytes) return fail(HM_EINVAL, "NULL argument");
    *bytes = bond_corr_bytes(b, n_bonds);
    return HM_OK;
}

int bond_corr(const hm_basis *b, int n_bonds, const int32_t *u, const int32_t *v, const void *g,
              const void *x, double *out, int dtype, void *work, size_t work_bytes, void *stream) {
    if (!b) return fail(HM_EINVAL, "basis is NULL");
    if (dtype != HM_F64 && dtype != HM_F32) return fail(HM_EINVAL, "dtype must be HM_F64 or HM_F32");
    if (!g || !x || (n_bonds > 0 && !out)) return fail(HM_EINVAL, "NULL vector");
    std::vector<double> ones(n_bonds > 0 ? n_bonds : 1, 1.0);
    BondParams bp;
    HM_TRY(make_bonds(b, n_bonds, u, v, ones.data(), &bp));
    return bond_corr_dev(b, bp, g, x, out, dtype, work, work_bytes, 1.0, nullptr, as_stream(stream));
}

int start_vector(const hm_basis *b, uint64_t seed, int kind, void *x, int dtype, void *stream) {
    if (!b || !x) return fail(HM_EINVAL, "NULL argument");
    if (kind != 0 && kind != 1) return fail(HM_EINVAL, "kind must be 0 or 1");
    if (dtype != HM_F64 && dtype != HM_F32) return fail(HM_EINVAL, "bad dtype");
    return start_vector_dev(b->view.dim, seed, kind, x, dtype, as_stream(stream));
}

}  // extern "C"
