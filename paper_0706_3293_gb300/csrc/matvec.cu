// matvec.cu -- y = H x by rows (Eq. E-4-b), the bond-correlation adjoint, start vectors.
#include <algorithm>
#include <cstdio>
#include <mutex>

#include "hm_row.cuh"
#include "s1blk.cuh"

namespace hm {

// ---------------------------------------------------------------------------------------
// general row kernel: one thread per output row, grid-stride over rows
// ---------------------------------------------------------------------------------------
template <class I, class T, class Acc, int NV>
__global__ void __launch_bounds__(256)
k_matvec(SectorView sv, BondParams bp, const T *__restrict__ x, T *__restrict__ y, int ld, int c0, int run) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    const double *pdn, *pup;
    const I *cd = stage_tables<I>(sv, bp, smem_raw, &pdn, &pup);
    I *const px = row_px_base<I>(sv, smem_raw);
    Codec<I> c{cd, sv.N, sv.S2, sv.A, sv.bits, sv.cd_w, sv.cd_rowlen};
    row_runs(c, sv.dim, px, run, [&](uint64_t r, uint64_t w) {
        const I i = (I)r;
        Acc acc[NV], dg;
        row_apply<I, T, Acc, NV>(c, bp, pdn, pup, i, w, x, ld, c0, acc, &dg, px);
        const T *xi = x + r * ld + c0;
        T *yi = y + r * ld + c0;
#pragma unroll
        for (int k = 0; k < NV; ++k) yi[k] = (T)(dg * (Acc)xi[k] + acc[k]);
    });
}

template <class I, class T, class Acc, int NV>
static int launch_matvec(const SectorView &sv, const BondParams &bp, const T *x, T *y, int ld,
                         int c0, cudaStream_t st) {
    size_t sm = row_smem_bytes<I>(sv);
    HM_CUDA(raise_smem_limit(k_matvec<I, T, Acc, NV>, (int)sm));
    k_matvec<I, T, Acc, NV><<<grid_blocks(sv.dim, 256), 256, sm, st>>>(sv, bp, x, y, ld, c0, row_run_len());
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
    HM_CUDA(raise_smem_limit(k_bond_corr<I, T>, (int)sm));
    dim3 grid(nblk, (bp.nb + BC - 1) / BC);
    k_bond_corr<I, T><<<grid, 256, sm, st>>>(sv, bp, g, x, part);
    HM_CUDA(cudaGetLastError());
    k_reduce_rows<<<bp.nb < 1024 ? bp.nb : 1024, 256, 0, st>>>(part, nblk, bp.nb, sign, div, out);
    HM_CUDA(cudaGetLastError());
    return HM_OK;
}

int blk_bond_corr(hm_basis *b, const BondParams &bp, const void *g, const void *x, double *out, int dtype,
                  void *work, size_t work_bytes, double sign, const double *div, cudaStream_t st);
size_t blk_bond_corr_bytes();

// general row kernels of bond_corr (any s, no per-basis tables beyond the basis's own and no
// run-time compilation); part: nblk x n_bonds doubles
static int bond_corr_rows(const SectorView &sv, const BondParams &bp, const void *g, const void *x, double *out,
                          int dtype, double *part, int nblk, double sign, const double *div, cudaStream_t st) {
    if (dtype == HM_F64) {
        if (sv.idx64) return bond_corr_t<uint64_t, double>(sv, bp, (const double *)g, (const double *)x, out, part, nblk, sign, div, st);
        return bond_corr_t<uint32_t, double>(sv, bp, (const double *)g, (const double *)x, out, part, nblk, sign, div, st);
    }
    if (sv.idx64) return bond_corr_t<uint64_t, float>(sv, bp, (const float *)g, (const float *)x, out, part, nblk, sign, div, st);
    return bond_corr_t<uint32_t, float>(sv, bp, (const float *)g, (const float *)x, out, part, nblk, sign, div, st);
}

int bond_corr_dev(const hm_basis *b, const BondParams &bp, const void *g, const void *x,
                  double *out, int dtype, void *work, size_t work_bytes, double sign,
                  const double *div, cudaStream_t st) {
    const SectorView &sv = b->view;
    const int nblk = grid_blocks(sv.dim, 256);
    if (bp.nb == 0) return HM_OK;
    // s = 1/2 sectors: the block kernels compiled per chunk of bonds (blk.cu)
    const int brc = blk_bond_corr(const_cast<hm_basis *>(b), bp, g, x, out, dtype, work, work_bytes, sign, div, st);
    if (brc <= 0) return brc;
    if (!work || work_bytes < (size_t)nblk * bp.nb * sizeof(double))
        return fail(HM_EWORKSPACE, "bond_corr needs %zu workspace bytes",
                    (size_t)nblk * bp.nb * sizeof(double));
    return bond_corr_rows(sv, bp, g, x, out, dtype, (double *)work, nblk, sign, div, st);
}

size_t bond_corr_bytes(const hm_basis *b, int n_bonds) {
    const size_t gen = (size_t)grid_blocks(b->view.dim, 256) * (size_t)(n_bonds > 0 ? n_bonds : 1) * sizeof(double);
    return std::max(gen, blk_bond_corr_bytes());
}

int blk_matvec(hm_basis *b, const BondParams &bp, const void *x, void *y, int dtype, int nvec,
               cudaStream_t st);
const char *blk_matvec_kernel(hm_basis *b, const BondParams &bp, int dtype, int nvec);

int matvec_dev(const hm_basis *b, const BondParams &bp, const void *x, void *y, int dtype,
               int nvec, cudaStream_t st) {
    const SectorView &sv = b->view;
    if (b->mom_k >= 0) {
        if (nvec != 1) return fail(HM_EINVAL, "momentum basis: one vector per product");
        return mom_matvec(b, bp, x, y, dtype, st);
    }
    // s = 1/2 sectors with few coupling classes take the block path (blk.cu)
    const int brc = blk_matvec(const_cast<hm_basis *>(b), bp, x, y, dtype, nvec, st);
    if (brc <= 0) return brc;
    // s = 1 FP32 products: the block kernel of s1blk.cu
    if (dtype == HM_F32 && nvec == 1 && sv.S2 == 2) {
        S1Plan P;
        const int src = s1_plan(const_cast<hm_basis *>(b), bp, &P);
        if (src < 0) return src;
        if (src == 0) return s1_matvec(P, (const float *)x, (float *)y, st);
    }
    if (b->parity)
        return fail(HM_EINVAL, "spin-flip basis: this bond list or vector count does not take the s = 1/2 block path");
    if (dtype == HM_F64) {
        if (sv.idx64) return matvec_cols<uint64_t, double, double>(sv, bp, (const double *)x, (double *)y, nvec, st);
        return matvec_cols<uint32_t, double, double>(sv, bp, (const double *)x, (double *)y, nvec, st);
    }
    if (sv.idx64) return matvec_cols<uint64_t, float, float>(sv, bp, (const float *)x, (float *)y, nvec, st);
    return matvec_cols<uint32_t, float, float>(sv, bp, (const float *)x, (float *)y, nvec, st);
}

// ---------------------------------------------------------------------------------------
// number of non-zero matrix elements: one diagonal per row plus every allowed exchange
// ---------------------------------------------------------------------------------------
template <class I>
__global__ void __launch_bounds__(256)
k_count_nnz(SectorView sv, BondParams bp, unsigned long long *out) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    const double *pdn, *pup;
    const I *cd = stage_tables<I>(sv, bp, smem_raw, &pdn, &pup);
    Codec<I> c{cd, sv.N, sv.S2, sv.A, sv.bits, sv.cd_w, sv.cd_rowlen};
    unsigned long long cnt = 0;
    for (uint64_t r = blockIdx.x * (uint64_t)blockDim.x + threadIdx.x; r < sv.dim;
         r += (uint64_t)gridDim.x * blockDim.x) {
        const uint64_t w = c.decode((I)r);
        cnt += 1;
        for (int t = 0; t < bp.nb; ++t) {
            const int ap = dig(w, bp.p[t], sv.bits), aq = dig(w, bp.q[t], sv.bits);
            cnt += (ap >= 1 && aq < sv.S2) + (ap < sv.S2 && aq >= 1);
        }
    }
    for (int o = 16; o > 0; o >>= 1) cnt += __shfl_down_sync(0xffffffffu, cnt, o);
    if ((threadIdx.x & 31) == 0) atomicAdd(out, cnt);   // integer sum: order-independent
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

int matvec_kernel_name(const hm_basis *b, int n_bonds, const int32_t *u, const int32_t *v, const double *J,
                       int dtype, int nvec, char *name, int cap) {
    if (!b || !name || cap < 1) return fail(HM_EINVAL, "NULL argument");
    if (dtype != HM_F64 && dtype != HM_F32) return fail(HM_EINVAL, "dtype must be HM_F64 or HM_F32");
    BondParams bp;
    HM_TRY(make_bonds(b, n_bonds, u, v, J, &bp));
    if (b->mom_k >= 0) {
        snprintf(name, (size_t)cap, "%s", "k_mom_matvec");
        return HM_OK;
    }
    const char *n = blk_matvec_kernel(const_cast<hm_basis *>(b), bp, dtype, nvec);
    if (!n && dtype == HM_F32 && nvec == 1 && b->view.S2 == 2) {
        S1Plan P;
        const int src = s1_plan(const_cast<hm_basis *>(b), bp, &P);
        if (src < 0) return src;
        if (src == 0) n = s1_kernel_name(P, 0);
    }
    if (!n && b->parity) return fail(HM_EINVAL, "spin-flip basis: this bond list or vector count does not take the s = 1/2 block path");
    snprintf(name, (size_t)cap, "%s", n ? n : "k_matvec");
    return HM_OK;
}

int count_nnz(const hm_basis *b, int n_bonds, const int32_t *u, const int32_t *v, int64_t *nnz,
              void *stream) {
    if (b && b->parity) return fail(HM_EINVAL, "count_nnz: not available on a spin-flip basis");
    if (!b || !nnz) return fail(HM_EINVAL, "NULL argument");
    std::vector<double> ones(n_bonds > 0 ? n_bonds : 1, 1.0);
    BondParams bp;
    HM_TRY(make_bonds(b, n_bonds, u, v, ones.data(), &bp));
    if (b->mom_k >= 0) return mom_count_nnz(b, bp, nnz, as_stream(stream));
    const SectorView &sv = b->view;
    cudaStream_t st = as_stream(stream);
    HM_CUDA(cudaMemsetAsync(nnz, 0, sizeof(int64_t), st));
    if (sv.idx64) {
        const size_t sm = row_smem_bytes<uint64_t>(sv);
        HM_CUDA(raise_smem_limit(k_count_nnz<uint64_t>, (int)sm));
        k_count_nnz<uint64_t><<<grid_blocks(sv.dim, 256), 256, sm, st>>>(sv, bp, (unsigned long long *)nnz);
    } else {
        const size_t sm = row_smem_bytes<uint32_t>(sv);
        HM_CUDA(raise_smem_limit(k_count_nnz<uint32_t>, (int)sm));
        k_count_nnz<uint32_t><<<grid_blocks(sv.dim, 256), 256, sm, st>>>(sv, bp, (unsigned long long *)nnz);
    }
    HM_CUDA(cudaGetLastError());
    return HM_OK;
}

int bond_corr_workspace(const hm_basis *b, int n_bonds, size_t *bytes) {
    if (!b || !bytes) return fail(HM_EINVAL, "NULL argument");
    *bytes = bond_corr_bytes(b, n_bonds);
    return HM_OK;
}

int bond_corr(const hm_basis *b, int n_bonds, const int32_t *u, const int32_t *v, const void *g,
              const void *x, double *out, int dtype, void *work, size_t work_bytes, void *stream) {
    if (b && b->parity) return fail(HM_EINVAL, "bond_corr: not available on a spin-flip basis");
    if (b && b->mom_k >= 0) return fail(HM_EINVAL, "bond_corr: not available on a momentum basis");
    if (!b) return fail(HM_EINVAL, "basis is NULL");
    if (dtype != HM_F64 && dtype != HM_F32) return fail(HM_EINVAL, "dtype must be HM_F64 or HM_F32");
    if (!g || !x || (n_bonds > 0 && !out)) return fail(HM_EINVAL, "NULL vector");
    std::vector<double> ones(n_bonds > 0 ? n_bonds : 1, 1.0);
    BondParams bp;
    HM_TRY(make_bonds(b, n_bonds, u, v, ones.data(), &bp));
    return bond_corr_dev(b, bp, g, x, out, dtype, work, work_bytes, 1.0, nullptr, as_stream(stream));
}

// ---- bond correlations without allocation ----------------------------------------------------
// Some callers cannot call cudaMalloc at the point where they need the adjoint: a host
// program that reserves its whole device-memory budget at start-up and forbids any later
// allocation (so that a long N = 32 run, whose Lanczos vectors fill most of the GPU, can
// never fail half-way for want of memory), or a library embedded in a framework whose own
// allocator owns all device memory and whose rules forbid side allocations.  For them
// bond_corr_static keeps its per-block partial sums in this file-scope device array and
// runs only the general row kernels, which read nothing but the basis's own tables (made
// by basis_build): no block tables built on first use, no run-time compiled kernel.
constexpr size_t HM_BC_STATIC_DOUBLES = 131072;   // 1 MiB on every device that loads the library
static __device__ __align__(256) double g_bc_static[HM_BC_STATIC_DOUBLES];

namespace {
constexpr int HM_BC_MAX_DEVICES = 64;
std::mutex g_bc_mutex;
struct BcStaticAddr {
    unsigned long long ctx_id;          // CUDA context the address belongs to (0: none yet)
    double *ptr;                        // device address of g_bc_static in that context
};
BcStaticAddr g_bc_addr[HM_BC_MAX_DEVICES];

// ID of the current context (cuCtxGetId through the runtime's driver entry point, so the
// library needs no link against libcuda); 0 when it cannot be read
unsigned long long current_ctx_id() {
    using Fn = int (*)(void *, unsigned long long *);
    static Fn fn = [] {
        void *p = nullptr;
        cudaDriverEntryPointQueryResult q;
        if (cudaGetDriverEntryPointByVersion("cuCtxGetId", &p, 12000, cudaEnableDefault, &q) != cudaSuccess ||
            q != cudaDriverEntryPointSuccess) {
            cudaGetLastError();
            return (Fn) nullptr;
        }
        return (Fn)p;
    }();
    unsigned long long id = 0;
    if (!fn || fn(nullptr, &id) != 0) return 0;
    return id;
}

// The host-side name g_bc_static is only a stand-in for the array: a kernel given it would
// fault, or silently use the wrong memory where the GPU can reach host memory.  Kernels need
// the device address, which cudaGetSymbolAddress gives (it allocates nothing).  It is looked
// up once per device, with that device current, on the first call there; a new context on
// the device (after cudaDeviceReset) is noticed by its ID and the address is looked up again.
int bc_static_ptr(double **out) {
    int dev = 0;
    HM_CUDA(cudaGetDevice(&dev));
    if (dev < 0 || dev >= HM_BC_MAX_DEVICES) return fail(HM_EINVAL, "device index %d out of range", dev);
    const unsigned long long id = current_ctx_id();
    std::lock_guard<std::mutex> lk(g_bc_mutex);
    BcStaticAddr &a = g_bc_addr[dev];
    if (!a.ptr || id == 0 || a.ctx_id != id) {
        void *p = nullptr;
        cudaError_t e = cudaGetSymbolAddress(&p, g_bc_static);
        if (e != cudaSuccess) return cuda_fail(e, "cudaGetSymbolAddress(g_bc_static)");
        a.ptr = (double *)p;
        a.ctx_id = id;
    }
    *out = a.ptr;
    return HM_OK;
}
}  // namespace

int bond_corr_static(const hm_basis *b, int n_bonds, const int32_t *u, const int32_t *v, const void *g,
                     const void *x, double *out, int dtype, void *stream) {
    if (b && b->parity) return fail(HM_EINVAL, "bond_corr: not available on a spin-flip basis");
    if (b && b->mom_k >= 0) return fail(HM_EINVAL, "bond_corr: not available on a momentum basis");
    if (!b) return fail(HM_EINVAL, "basis is NULL");
    if (dtype != HM_F64 && dtype != HM_F32) return fail(HM_EINVAL, "dtype must be HM_F64 or HM_F32");
    if (!g || !x || (n_bonds > 0 && !out)) return fail(HM_EINVAL, "NULL vector");
    if (n_bonds < 0 || n_bonds > HM_MAX_BONDS) return fail(HM_EINVAL, "n_bonds must be in 0..%d", HM_MAX_BONDS);
    double ones[HM_MAX_BONDS];
    for (int t = 0; t < n_bonds; ++t) ones[t] = 1.0;
    BondParams bp;
    HM_TRY(make_bonds(b, n_bonds, u, v, ones, &bp));
    if (bp.nb == 0) return HM_OK;
    // the general kernels' partial sums: grid_blocks x n_bonds doubles
    const int nblk = grid_blocks(b->view.dim, 256);
    const size_t need = (size_t)nblk * bp.nb * sizeof(double);
    if (need > HM_BC_STATIC_DOUBLES * sizeof(double))
        return fail(HM_EINVAL, "bond_corr_static: %zu bytes of partial sums exceed the %zu-byte static "
                    "scratch (fewer bonds or bond_corr with a workspace)", need,
                    HM_BC_STATIC_DOUBLES * sizeof(double));
    double *scratch = nullptr;
    HM_TRY(bc_static_ptr(&scratch));
    // every slot the reduction reads is written by this call's first kernel: nothing in the
    // shared array has to start at zero
    return bond_corr_rows(b->view, bp, g, x, out, dtype, scratch, nblk, 1.0, nullptr, as_stream(stream));
}

int start_vector(const hm_basis *b, uint64_t seed, int kind, void *x, int dtype, void *stream) {
    if (!b || !x) return fail(HM_EINVAL, "NULL argument");
    if (kind != 0 && kind != 1) return fail(HM_EINVAL, "kind must be 0 or 1");
    if (dtype != HM_F64 && dtype != HM_F32) return fail(HM_EINVAL, "bad dtype");
    return start_vector_dev(b->view.dim, seed, kind, x, dtype, as_stream(stream));
}

}  // extern "C"
