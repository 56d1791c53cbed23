// basis.cu -- sector tables (Sec. 3, Eq. E-3-c), the codec test hooks (Sec. 3.1, 3.2),
// bond preparation, seeded start vectors and error reporting.
#include <stdlib.h>
#include <cmath>
#include <cstdarg>
#include <cstdio>
#include <cstring>
#include <new>

#include "hm_internal.cuh"

namespace hm {

static thread_local std::string g_err;

int fail(int code, const char *fmt, ...) {
    char buf[512];
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(buf, sizeof buf, fmt, ap);
    va_end(ap);
    g_err = buf;
    return code;
}

int cuda_fail(cudaError_t e, const char *what) {
    return fail(HM_ECUDA, "%s: %s (%s)", what, cudaGetErrorString(e), cudaGetErrorName(e));
}

cudaStream_t as_stream(void *s) { return reinterpret_cast<cudaStream_t>(s); }

int digit_bits(int two_s) { return two_s == 1 ? 1 : (two_s <= 3 ? 2 : 4); }

int check_sector(int n_sites, int two_s, int two_m, int *A) {
    if (two_s < 1 || two_s > 7) return fail(HM_EINVAL, "two_s must be in 1..7 (got %d)", two_s);
    if (n_sites < 1 || n_sites > HM_MAX_SITES)
        return fail(HM_EINVAL, "n_sites must be in 1..%d (got %d)", HM_MAX_SITES, n_sites);
    if (n_sites * digit_bits(two_s) > 64)
        return fail(HM_EINVAL, "n_sites * bits-per-digit exceeds 64 (N=%d, 2s=%d)", n_sites, two_s);
    long t = (long)n_sites * two_s - two_m;
    if (t % 2 != 0 || t < 0 || t > 2L * n_sites * two_s)
        return fail(HM_EPARITY, "2M=%d is not a magnetic quantum number of N=%d spins 2s=%d",
                    two_m, n_sites, two_s);
    *A = (int)(t / 2);
    return HM_OK;
}

// D(k, a) by Eq. (E-3-c) and CD[p][S][a] = sum_{n<a} D(p, S-n); entries of rows
// (p, S) that no sector state reaches are stored as 0.
int build_tables(int n_sites, int two_s, int two_m, hm_basis *b) {
    int A = 0;
    HM_TRY(check_sector(n_sites, two_s, two_m, &A));
    const int N = n_sites, S2 = two_s, W = S2 * N + 1;
    const uint64_t LIM = 1ull << 63;
    b->D.assign((size_t)(N + 1) * W, 0);
    auto D = [&](int k, int a) -> uint64_t {
        if (k < 0 || k > N || a < 0 || a > S2 * k) return 0;
        return b->D[(size_t)k * W + a];
    };
    b->D[0] = 1;
    for (int k = 1; k <= N; ++k)
        for (int a = 0; a <= S2 * k; ++a) {
            uint64_t s = 0;
            for (int n = 0; n <= S2; ++n) {
                s += D(k - 1, a - n);
                if (s >= LIM) return fail(HM_EOVERFLOW, "D(%d,%d) exceeds 2^63", k, a);
            }
            b->D[(size_t)k * W + a] = s;
        }
    const uint64_t dim = D(N, A);
    SectorView &v = b->view;
    v.N = N; v.S2 = S2; v.A = A; v.bits = digit_bits(S2);
    v.cd_w = S2 + 2;
    v.cd_rowlen = (A + 1) * v.cd_w;
    v.cd_len = N * v.cd_rowlen;
    v.dim = dim;
    v.idx64 = dim >= (1ull << 32) ? 1 : 0;
    v.cd = nullptr;
    b->cd.assign((size_t)v.cd_len, 0);
    for (int p = 0; p < N; ++p)
        for (int S = 0; S <= A; ++S) {
            bool reach = S <= S2 * (p + 1) && (A - S) <= S2 * (N - 1 - p);
            if (!reach) continue;
            uint64_t c = 0;
            for (int a = 0; a <= S2 + 1; ++a) {
                b->cd[(size_t)p * v.cd_rowlen + S * v.cd_w + a] = c;
                if (a <= S2) c += D(p, S - a);
            }
            if (c > dim) return fail(HM_EOVERFLOW, "rank table entry above the dimension");
        }
    return HM_OK;
}

int sm_count() {
    static int n = 0;
    if (n == 0) {
        int dev = 0;
        cudaGetDevice(&dev);
        if (cudaDeviceGetAttribute(&n, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess || n <= 0)
            n = 1;
    }
    return n;
}

int grid_blocks(uint64_t rows, int threads) {
    uint64_t need = (rows + threads - 1) / threads;
    uint64_t cap = (uint64_t)sm_count() * 8;
    if (need < 1) need = 1;
    return (int)(need < cap ? need : cap);
}

int row_run_len() {
    const char *e = getenv("HM_ROW_RUN");
    const int v = e ? atoi(e) : 1;
    return v < 1 ? 1 : v > 64 ? 64 : v;
}

int make_bonds(const hm_basis *b, int n_bonds, const int32_t *u, const int32_t *v,
               const double *J, BondParams *out) {
    HM_TRY(bonds_check(b->view.N, n_bonds, u, v, J));
    const int S2 = b->view.S2;
    out->nb = n_bonds;
    out->S2 = S2;
    for (int t = 0; t < n_bonds; ++t) {
        int p = u[t], q = v[t];
        if (p > q) { int s = p; p = q; q = s; }   // s_u.s_v is symmetric in u, v
        out->p[t] = (unsigned char)p;
        out->q[t] = (unsigned char)q;
        out->jm[t] = -J[t];
        out->jmf[t] = (float)(-J[t]);
    }
    for (int ap = 0; ap <= S2; ++ap)
        for (int aq = 0; aq <= S2; ++aq) {
            long up_p = (long)ap * (S2 - ap + 1), dn_p = (long)(S2 - ap) * (ap + 1);
            long up_q = (long)aq * (S2 - aq + 1), dn_q = (long)(S2 - aq) * (aq + 1);
            out->hs_pdn[ap * 8 + aq] = 0.5 * std::sqrt((double)(up_p * dn_q));
            out->hs_pup[ap * 8 + aq] = 0.5 * std::sqrt((double)(dn_p * up_q));
        }
    if (b->mom_k >= 0) HM_TRY(mom_check_bonds(b, n_bonds, u, v, J));
    return HM_OK;
}

// ---------------------------------------------------------------------------------------
// codec test hooks
// ---------------------------------------------------------------------------------------
template <class I>
__global__ void k_decode(SectorView sv, const int64_t *__restrict__ idx,
                         uint64_t *__restrict__ out, int64_t n) {
    extern __shared__ unsigned char smem_raw[];
    I *cd = reinterpret_cast<I *>(smem_raw);
    for (int k = threadIdx.x; k < sv.cd_len; k += blockDim.x) cd[k] = ((const I *)sv.cd)[k];
    __syncthreads();
    Codec<I> c{cd, sv.N, sv.S2, sv.A, sv.bits, sv.cd_w, sv.cd_rowlen};
    for (int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; t < n;
         t += (int64_t)gridDim.x * blockDim.x) {
        int64_t i = idx[t];
        out[t] = (i < 0 || (uint64_t)i >= sv.dim) ? ~0ull : c.decode((I)i);
    }
}

template <class I>
__global__ void k_encode(SectorView sv, const uint64_t *__restrict__ st,
                         int64_t *__restrict__ out, int64_t n) {
    extern __shared__ unsigned char smem_raw[];
    I *cd = reinterpret_cast<I *>(smem_raw);
    for (int k = threadIdx.x; k < sv.cd_len; k += blockDim.x) cd[k] = ((const I *)sv.cd)[k];
    __syncthreads();
    Codec<I> c{cd, sv.N, sv.S2, sv.A, sv.bits, sv.cd_w, sv.cd_rowlen};
    for (int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; t < n;
         t += (int64_t)gridDim.x * blockDim.x) {
        uint64_t w = st[t];
        // validity: digits <= 2s, no bits above the N positions, digit sum A
        bool ok = (sv.N * sv.bits >= 64) || (w >> (sv.N * sv.bits)) == 0;
        int S = 0;
        for (int p = 0; p < sv.N && ok; ++p) {
            int a = dig(w, p, sv.bits);
            if (a > sv.S2) ok = false;
            S += a;
        }
        ok = ok && S == sv.A;
        const int64_t ix = ok ? (int64_t)c.encode(w) : -1;
        out[t] = ix >= 0 && (uint64_t)ix < sv.dim ? ix : -1;   // spin-flip basis: representatives only
    }
}

template <class I>
static size_t cd_bytes(const SectorView &sv) { return (size_t)sv.cd_len * sizeof(I); }

}  // namespace hm

using namespace hm;

extern "C" {

const char *hm_last_error(void) { return g_err.c_str(); }

int basis_dim_query(int n_sites, int two_s, int two_m, int64_t *dim) {
    if (!dim) return fail(HM_EINVAL, "dim is NULL");
    hm_basis tmp;
    HM_TRY(build_tables(n_sites, two_s, two_m, &tmp));
    *dim = (int64_t)tmp.view.dim;
    return HM_OK;
}

int bonds_check(int n_sites, int n_bonds, const int32_t *u, const int32_t *v, const double *J) {
    if (n_bonds < 0 || n_bonds > HM_MAX_BONDS)
        return fail(HM_EINVAL, "n_bonds must be in 0..%d (got %d)", HM_MAX_BONDS, n_bonds);
    if (n_bonds > 0 && (!u || !v || !J)) return fail(HM_EINVAL, "bond arrays are NULL");
    for (int t = 0; t < n_bonds; ++t) {
        if (u[t] < 0 || u[t] >= n_sites || v[t] < 0 || v[t] >= n_sites)
            return fail(HM_EINVAL, "bond %d (%d,%d) outside 0..%d", t, u[t], v[t], n_sites - 1);
        if (u[t] == v[t]) return fail(HM_EINVAL, "bond %d joins site %d to itself", t, u[t]);
        if (!std::isfinite(J[t])) return fail(HM_EINVAL, "bond %d has a non-finite coupling", t);
    }
    return HM_OK;
}

int basis_build(int n_sites, int two_s, int two_m, hm_basis **out) {
    if (!out) return fail(HM_EINVAL, "out is NULL");
    *out = nullptr;
    hm_basis *b = new (std::nothrow) hm_basis();
    if (!b) return fail(HM_ENOMEM, "host allocation failed");
    int rc = build_tables(n_sites, two_s, two_m, b);
    if (rc < 0) { delete b; return rc; }
    SectorView &v = b->view;
    size_t bytes = v.idx64 ? (size_t)v.cd_len * 8 : (size_t)v.cd_len * 4;
    std::vector<uint32_t> c32;
    const void *src = b->cd.data();
    if (!v.idx64) {
        c32.resize(v.cd_len);
        for (int k = 0; k < v.cd_len; ++k) c32[k] = (uint32_t)b->cd[k];
        src = c32.data();
    }
    cudaError_t e = cudaGetDevice(&b->device);
    if (e == cudaSuccess) e = cudaMalloc(&b->d_cd, bytes > 0 ? bytes : 8);
    if (e == cudaSuccess) e = cudaMalloc(&b->d_scratch, 256);
    if (e == cudaSuccess) e = cudaMemcpy(b->d_cd, src, bytes, cudaMemcpyHostToDevice);
    if (e != cudaSuccess) {
        if (b->d_cd) cudaFree(b->d_cd);
        if (b->d_scratch) cudaFree(b->d_scratch);
        delete b;
        return cuda_fail(e, "basis_build: device tables");
    }
    v.cd = b->d_cd;
    *out = b;
    return HM_OK;
}

int basis_build_flip(int n_sites, int parity, hm_basis **out) {
    if (!out) return fail(HM_EINVAL, "out is NULL");
    *out = nullptr;
    if (parity != 1 && parity != -1) return fail(HM_EINVAL, "parity must be +1 or -1 (got %d)", parity);
    if (n_sites < 10 || n_sites > 32 || (n_sites & 1))
        return fail(HM_EINVAL, "spin-flip basis needs an even n_sites in 10..32 (got %d)", n_sites);
    HM_TRY(basis_build(n_sites, 1, 0, out));
    (*out)->parity = parity;
    (*out)->view.dim /= 2;          // the representatives: the first half of the sector
    return HM_OK;
}

int basis_free(hm_basis *b) {
    if (!b) return HM_OK;
    cudaError_t e = cudaSuccess, e2;
    if (b->d_cd && (e2 = cudaFree(b->d_cd)) != cudaSuccess) e = e2;
    if (b->d_scratch && (e2 = cudaFree(b->d_scratch)) != cudaSuccess) e = e2;
    for (auto &kv : b->blk_tabs)
        if (kv.second.dev && (e2 = cudaFree(kv.second.dev)) != cudaSuccess) e = e2;
    for (auto &kv : b->s1_tabs)
        if (kv.second.dev && (e2 = cudaFree(kv.second.dev)) != cudaSuccess) e = e2;
    for (auto &kv : b->blk_ttabs)
        if (kv.second && (e2 = cudaFree(kv.second)) != cudaSuccess) e = e2;
    if (b->d_mom && (e2 = cudaFree(b->d_mom)) != cudaSuccess) e = e2;
    delete b;
    if (e != cudaSuccess) return cuda_fail(e, "basis_free");
    return HM_OK;
}

int basis_dim(const hm_basis *b, int64_t *dim) {
    if (!b || !dim) return fail(HM_EINVAL, "NULL argument");
    *dim = (int64_t)b->view.dim;
    return HM_OK;
}

int basis_decode(const hm_basis *b, const int64_t *idx, uint64_t *states, int64_t n, void *stream) {
    if (!b || n < 0 || (n > 0 && (!idx || !states))) return fail(HM_EINVAL, "bad argument");
    if (b->mom_k >= 0) return fail(HM_EINVAL, "basis_decode: not available on a momentum basis");
    if (n == 0) return HM_OK;
    const SectorView &sv = b->view;
    int blocks = grid_blocks((uint64_t)n, 256);
    if (sv.idx64) {
        size_t sm = cd_bytes<uint64_t>(sv);
        HM_CUDA(raise_smem_limit(k_decode<uint64_t>, (int)sm));
        k_decode<uint64_t><<<blocks, 256, sm, as_stream(stream)>>>(sv, idx, states, n);
    } else {
        size_t sm = cd_bytes<uint32_t>(sv);
        HM_CUDA(raise_smem_limit(k_decode<uint32_t>, (int)sm));
        k_decode<uint32_t><<<blocks, 256, sm, as_stream(stream)>>>(sv, idx, states, n);
    }
    HM_CUDA(cudaGetLastError());
    return HM_OK;
}

int basis_encode(const hm_basis *b, const uint64_t *states, int64_t *idx, int64_t n, void *stream) {
    if (!b || n < 0 || (n > 0 && (!idx || !states))) return fail(HM_EINVAL, "bad argument");
    if (b->mom_k >= 0) return fail(HM_EINVAL, "basis_encode: not available on a momentum basis");
    if (n == 0) return HM_OK;
    const SectorView &sv = b->view;
    int blocks = grid_blocks((uint64_t)n, 256);
    if (sv.idx64) {
        size_t sm = cd_bytes<uint64_t>(sv);
        HM_CUDA(raise_smem_limit(k_encode<uint64_t>, (int)sm));
        k_encode<uint64_t><<<blocks, 256, sm, as_stream(stream)>>>(sv, states, idx, n);
    } else {
        size_t sm = cd_bytes<uint32_t>(sv);
        HM_CUDA(raise_smem_limit(k_encode<uint32_t>, (int)sm));
        k_encode<uint32_t><<<blocks, 256, sm, as_stream(stream)>>>(sv, states, idx, n);
    }
    HM_CUDA(cudaGetLastError());
    return HM_OK;
}

}  // extern "C"
