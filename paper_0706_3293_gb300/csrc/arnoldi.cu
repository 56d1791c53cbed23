// arnoldi.cu -- the products of Eq. E-4-b under two other Krylov-type methods: Arnoldi
// with full re-orthogonalisation and the shifted power (projection) method.  The paper
// ports its product to such methods in its closing summary without giving them; the
// iterations below are the textbook ones (Arnoldi 1951; classical Gram-Schmidt applied
// twice, Giraud, Langou and Rozloznik 2005; the power method on sigma - H).
//
// FP64 vectors, one vector per product, every step enqueued on the caller's stream with
// no host round trip: the scalars (h, beta, energies, the stop flag) stay on the device.
// Reductions run over a fixed grid in a fixed order, so every run is reproducible.
// The Arnoldi basis is kept as double-float pairs (47 significant bits, relative error
// below 2^-46) and the Gram-Schmidt dots and updates run in double-float arithmetic on
// the FP32 pipe: binary64 multiply-adds run at a small fraction of that rate on this GPU
// and bounded the first version (2.2 TB/s for the dots).
#include <algorithm>
#include <cmath>
#include <vector>

#include "ef64.cuh"
#include "hm_internal.cuh"

namespace hm {

int matvec_dev(const hm_basis *b, const BondParams &bp, const void *x, void *y, int dtype, int nvec,
               cudaStream_t st);
int start_vector_dev(uint64_t n, uint64_t seed, int kind, void *x, int dtype, cudaStream_t st);

namespace {

constexpr int AR_NT = 256;
constexpr int AR_RB = 4096;          // rows of a tile of k_mdot
constexpr int AR_MAXM = 1024;        // Arnoldi steps at most
constexpr double AR_TOL = 1e-12;     // breakdown: beta_j <= tol * max |H entries|

struct ArState {
    double scale;                    // max |H| entries so far
    double beta;                     // norm of the current residual
    int done;                        // 1 after a breakdown: later kernels return at once
    int steps;                       // columns of H completed
    int status;                      // < 0: zero start vector
};

size_t al256(size_t x) { return (x + 255) & ~(size_t)255; }

__device__ __forceinline__ ef::df ar_df(double v) { return ef::df_from_bits(ef::d2u(v), 0); }
__device__ __forceinline__ double ar_dbl(ef::df v) { return ef::u2d(ef::bits_from_df(v, 0)); }

// part[tile][i] = sum over the AR_RB rows of a tile of V_i[r] w[r] for every i < nv (ps:
// stride of a tile's partials).  The CTA stages its tile of w (as double-float pairs) in
// shared memory; warp k then streams the tile's slices of V_k, V_{k+8}, ... and reduces
// each by a fixed shuffle tree, so every vector slice and w are read once.
__global__ void __launch_bounds__(AR_NT) k_mdot(const float2 *__restrict__ V, size_t ldv, int nv,
                                                 const double *__restrict__ w, uint64_t n, double *__restrict__ part,
                                                 int ps, const ArState *__restrict__ st) {
    if (st->done) return;
    __shared__ float2 ws[AR_RB];
    const uint64_t r0 = (uint64_t)blockIdx.x * AR_RB;
    const int rows = (int)min((uint64_t)AR_RB, n - r0);
    for (int t = threadIdx.x; t < rows; t += AR_NT) {
        const ef::df d = ar_df(w[r0 + t]);
        ws[t] = make_float2(d.hi, d.lo);
    }
    __syncthreads();
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    for (int i = warp; i < nv; i += AR_NT / 32) {
        const float2 *vi = V + (size_t)i * ldv + r0;
        ef::df a0{0.0f, 0.0f}, a1{0.0f, 0.0f};
        int t = lane;
        for (; t + 32 < rows; t += 64) {                  // two independent chains
            const float2 v = vi[t], x = ws[t], v2 = vi[t + 32], x2 = ws[t + 32];
            a0 = ef::df_add(a0, ef::df_mul(ef::df{v.x, v.y}, ef::df{x.x, x.y}));
            a1 = ef::df_add(a1, ef::df_mul(ef::df{v2.x, v2.y}, ef::df{x2.x, x2.y}));
        }
        if (t < rows) {
            const float2 v = vi[t], x = ws[t];
            a0 = ef::df_add(a0, ef::df_mul(ef::df{v.x, v.y}, ef::df{x.x, x.y}));
        }
        double s = ((double)a0.hi + (double)a0.lo) + ((double)a1.hi + (double)a1.lo);
        for (int o = 16; o > 0; o >>= 1) s += __shfl_down_sync(0xffffffffu, s, o);
        if (lane == 0) part[(size_t)blockIdx.x * ps + i] = s;
    }
}

// h[i] = sum over blocks of part[blk][i] (fixed order), hcol[i] += h[i]: CTA i sums the
// partials of vector i
__global__ void __launch_bounds__(AR_NT) k_mdot_fin(const double *__restrict__ part, int nb, int ps,
                                                     double *__restrict__ h, double *__restrict__ hcol,
                                                     const ArState *__restrict__ st) {
    if (st->done) return;
    __shared__ double red[AR_NT / 32];
    const int i = blockIdx.x;
    double s = 0.0;
    for (int b = threadIdx.x; b < nb; b += AR_NT) s += part[(size_t)b * ps + i];
    s = block_sum<AR_NT>(s, red);
    if (threadIdx.x == 0) {
        h[i] = s;
        hcol[i] += s;
    }
}

// w[r] -= sum_{i < nv} h[i] V_i[r]  (double-float sum, w rounded back to binary64)
__global__ void __launch_bounds__(AR_NT) k_gs_sub(const float2 *__restrict__ V, size_t ldv, int nv,
                                                   const double *__restrict__ h, double *__restrict__ w, uint64_t n,
                                                   const ArState *__restrict__ st) {
    if (st->done) return;
    __shared__ float2 hs[AR_MAXM + 1];
    for (int i = threadIdx.x; i < nv; i += AR_NT) {
        const ef::df t = ar_df(-h[i]);
        hs[i] = make_float2(t.hi, t.lo);
    }
    __syncthreads();
    for (uint64_t r = (uint64_t)blockIdx.x * AR_NT + threadIdx.x; r < n; r += (uint64_t)gridDim.x * AR_NT) {
        ef::df s = ar_df(w[r]);
        for (int i = 0; i < nv; ++i) {
            const float2 v = V[(size_t)i * ldv + r], c = hs[i];
            s = ef::df_add(s, ef::df_mul(ef::df{c.x, c.y}, ef::df{v.x, v.y}));
        }
        w[r] = ar_dbl(s);
    }
}

// part[blk] = sum over the block's rows of a[r] b[r] (and of b[r]^2 into part2, if given)
__global__ void __launch_bounds__(AR_NT) k_dot2(const double *__restrict__ a, const double *__restrict__ b,
                                                 uint64_t n, double *__restrict__ part, double *__restrict__ part2,
                                                 const ArState *__restrict__ st) {
    if (st && st->done) return;
    __shared__ double red[AR_NT / 32];
    double s = 0.0, s2 = 0.0;
    for (uint64_t r = (uint64_t)blockIdx.x * AR_NT + threadIdx.x; r < n; r += (uint64_t)gridDim.x * AR_NT) {
        const double br = b[r];
        s = fma(a[r], br, s);
        s2 = fma(br, br, s2);
    }
    s = block_sum<AR_NT>(s, red);
    if (threadIdx.x == 0) part[blockIdx.x] = s;
    if (part2) {
        __syncthreads();
        s2 = block_sum<AR_NT>(s2, red);
        if (threadIdx.x == 0) part2[blockIdx.x] = s2;
    }
}

__device__ __forceinline__ double ar_sum(const double *__restrict__ part, int nb, double *red) {
    double s = 0.0;
    for (int b = threadIdx.x; b < nb; b += AR_NT) s += part[b];
    return block_sum<AR_NT>(s, red);       // valid in thread 0
}

// start: beta = |v|, status < 0 when it is zero
__global__ void __launch_bounds__(AR_NT) k_ar_start(const double *__restrict__ part, int nb, ArState *st) {
    __shared__ double red[AR_NT / 32];
    const double s = ar_sum(part, nb, red);
    if (threadIdx.x == 0) {
        st->scale = 0.0;
        st->steps = 0;
        st->beta = sqrt(s);
        st->done = s > 0.0 ? 0 : 1;
        st->status = s > 0.0 ? HM_OK : HM_EINVAL;
    }
}

// H[j+1, j] = beta_j = |w|; scale = max |H[:, j]|; breakdown when beta_j <= tol * scale
__global__ void __launch_bounds__(AR_NT) k_ar_beta(const double *__restrict__ part, int nb, double *__restrict__ hcol,
                                                    int j, ArState *st) {
    if (st->done) return;
    __shared__ double red[AR_NT / 32];
    const double s = ar_sum(part, nb, red);
    if (threadIdx.x == 0) {
        double sc = st->scale;
        for (int i = 0; i <= j; ++i) sc = fmax(sc, fabs(hcol[i]));
        const double beta = sqrt(s);
        hcol[j + 1] = beta;
        st->scale = fmax(sc, beta);
        st->beta = beta;
        st->steps = j + 1;
        if (beta <= AR_TOL * sc) st->done = 1;
    }
}

// next Krylov vector x / beta: into the basis (double-float) and, as binary64, into q,
// the input of the next product
__global__ void __launch_bounds__(AR_NT) k_ar_scale(const double *__restrict__ x, float2 *__restrict__ vout,
                                                     double *__restrict__ q, uint64_t n,
                                                     const ArState *__restrict__ st) {
    if (st->done) return;
    const double inv = 1.0 / st->beta;       // the scaled entries lie in double-float range
    for (uint64_t r = (uint64_t)blockIdx.x * AR_NT + threadIdx.x; r < n; r += (uint64_t)gridDim.x * AR_NT) {
        const double t = x[r] * inv;
        const ef::df d = ar_df(t);
        vout[r] = make_float2(d.hi, d.lo);
        q[r] = t;
    }
}

// Eigenvalues of a symmetric n x n matrix (row major, overwritten) by cyclic Jacobi
// rotations (Rutishauser's formulation), ascending into ev.
void jacobi_eigenvalues(std::vector<double> &a, int n, std::vector<double> &ev) {
    for (int sweep = 0; sweep < 100; ++sweep) {
        double off = 0.0, tot = 0.0;
        for (int p = 0; p < n; ++p)
            for (int q = 0; q < n; ++q) {
                tot += a[p * n + q] * a[p * n + q];
                if (p != q) off += a[p * n + q] * a[p * n + q];
            }
        if (off <= 1e-30 * tot || off == 0.0) break;
        for (int p = 0; p < n - 1; ++p)
            for (int q = p + 1; q < n; ++q) {
                const double apq = a[(size_t)p * n + q];
                if (apq == 0.0) continue;
                const double theta = (a[q * n + q] - a[p * n + p]) / (2.0 * apq);
                const double t = (theta >= 0 ? 1.0 : -1.0) / (std::fabs(theta) + std::sqrt(theta * theta + 1.0));
                const double c = 1.0 / std::sqrt(t * t + 1.0), s = t * c;
                for (int k = 0; k < n; ++k) {            // columns p, q
                    const double akp = a[k * n + p], akq = a[k * n + q];
                    a[k * n + p] = c * akp - s * akq;
                    a[k * n + q] = s * akp + c * akq;
                }
                for (int k = 0; k < n; ++k) {            // rows p, q
                    const double apk = a[p * n + k], aqk = a[q * n + k];
                    a[p * n + k] = c * apk - s * aqk;
                    a[q * n + k] = s * apk + c * aqk;
                }
            }
    }
    ev.resize(n);
    for (int i = 0; i < n; ++i) ev[i] = a[i * n + i];
    std::sort(ev.begin(), ev.end());
}

// ---- projection (shifted power) method ----------------------------------------------------
struct PrState {
    double inv;                      // 1 / |sigma psi - H psi| of the step
    int status;
};

// psi = v / |v|; status < 0 when v = 0
__global__ void __launch_bounds__(AR_NT) k_pr_start(const double *__restrict__ part, int nb, PrState *st) {
    __shared__ double red[AR_NT / 32];
    const double s = ar_sum(part, nb, red);
    if (threadIdx.x == 0) {
        st->inv = s > 0.0 ? 1.0 / sqrt(s) : 0.0;
        st->status = s > 0.0 ? HM_OK : HM_EINVAL;
    }
}

// E_k = psi . y (psi normalised), |sigma psi - y|^2 = sigma^2 - 2 sigma E_k + y . y
__global__ void __launch_bounds__(AR_NT) k_pr_fin(const double *__restrict__ p1, const double *__restrict__ p2, int nb,
                                                   double sigma, double *__restrict__ energy, PrState *st) {
    __shared__ double red[AR_NT / 32];
    const double e = ar_sum(p1, nb, red);
    __syncthreads();
    const double yy = ar_sum(p2, nb, red);
    if (threadIdx.x == 0) {
        *energy = e;
        const double nn = sigma * sigma - 2.0 * sigma * e + yy;
        st->inv = nn > 0.0 ? 1.0 / sqrt(nn) : 0.0;
    }
}

// psi = (sigma psi - y) * inv
__global__ void __launch_bounds__(AR_NT) k_pr_update(double *__restrict__ psi, const double *__restrict__ y, uint64_t n,
                                                      double sigma, const PrState *__restrict__ st) {
    const double inv = st->inv;
    for (uint64_t r = (uint64_t)blockIdx.x * AR_NT + threadIdx.x; r < n; r += (uint64_t)gridDim.x * AR_NT)
        psi[r] = (sigma * psi[r] - y[r]) * inv;
}

// psi = v * inv (start)
__global__ void __launch_bounds__(AR_NT) k_pr_scale(const double *__restrict__ v, double *__restrict__ psi, uint64_t n,
                                                     const PrState *__restrict__ st) {
    const double inv = st->inv;
    for (uint64_t r = (uint64_t)blockIdx.x * AR_NT + threadIdx.x; r < n; r += (uint64_t)gridDim.x * AR_NT)
        psi[r] = v[r] * inv;
}

struct ArLayout {
    size_t V, q, w, part, part2, h, H, st, total;
    size_t ldv;                      // elements between consecutive Krylov vectors
    int nb, ps;                      // blocks of the reductions, partials per block
    int nt;                          // row tiles of k_mdot
};

ArLayout ar_layout(uint64_t dim, int steps) {
    ArLayout L{};
    L.nb = grid_blocks(dim, AR_NT);
    L.ldv = al256(dim * 8) / 8;
    L.ps = steps + 1;
    size_t o = 0;
    L.V = o; o += (size_t)(steps + 1) * L.ldv * 8;
    L.q = o; o += al256(dim * 8);
    L.w = o; o += al256(dim * 8);
    L.nt = (int)((dim + AR_RB - 1) / AR_RB);
    L.part = o; o += al256((size_t)std::max(L.nb, L.nt) * L.ps * 8);
    L.part2 = o; o += al256((size_t)L.nb * 8);
    L.h = o; o += al256((size_t)(steps + 1) * 8);
    L.H = o; o += al256((size_t)(steps + 1) * steps * 8);
    L.st = o; o += al256(sizeof(ArState) + sizeof(PrState));
    L.total = o;
    return L;
}

}  // namespace
}  // namespace hm

using namespace hm;

extern "C" {

int arnoldi_workspace(const hm_basis *b, int steps, size_t *bytes) {
    if (!b || !bytes) return fail(HM_EINVAL, "NULL argument");
    if (steps < 1 || steps > AR_MAXM) return fail(HM_EINVAL, "steps must be in 1..%d", AR_MAXM);
    *bytes = ar_layout(b->view.dim, steps).total;
    return HM_OK;
}

int arnoldi_run(const hm_basis *b, int n_bonds, const int32_t *u, const int32_t *v, const double *J,
                const void *v0, uint64_t seed, int steps, void *work, size_t work_bytes, double *hess,
                int *steps_done, double *ritz, int n_ritz, void *stream) {
    if (!b || !steps_done) return fail(HM_EINVAL, "NULL argument");
    if (b->parity) return fail(HM_EINVAL, "arnoldi_run: not available on a spin-flip basis");
    if (steps < 1 || steps > AR_MAXM) return fail(HM_EINVAL, "steps must be in 1..%d", AR_MAXM);
    if (n_ritz < 0 || (n_ritz > 0 && !ritz)) return fail(HM_EINVAL, "bad n_ritz / ritz");
    BondParams bp;
    HM_TRY(make_bonds(b, n_bonds, u, v, J, &bp));
    const uint64_t dim = b->view.dim;
    const ArLayout L = ar_layout(dim, steps);
    if (!work || work_bytes < L.total || ((uintptr_t)work & 255))
        return fail(HM_EWORKSPACE, "workspace must be >= %zu bytes, 256-byte aligned", L.total);
    cudaStream_t st = as_stream(stream);
    unsigned char *W = (unsigned char *)work;
    float2 *V = (float2 *)(W + L.V);
    double *q = (double *)(W + L.q), *w = (double *)(W + L.w), *part = (double *)(W + L.part);
    double *h = (double *)(W + L.h), *H = (double *)(W + L.H);
    ArState *S = (ArState *)(W + L.st);
    const int nb = L.nb;
    HM_CUDA(cudaMemsetAsync(H, 0, (size_t)(steps + 1) * steps * 8, st));
    HM_CUDA(cudaMemsetAsync(S, 0, sizeof(ArState), st));
    // v_1 = v0 / |v0| (the seeded uniform vector when v0 is NULL)
    if (v0) HM_CUDA(cudaMemcpyAsync(w, v0, dim * 8, cudaMemcpyDeviceToDevice, st));
    else HM_TRY(start_vector_dev(dim, seed, 0, w, HM_F64, st));
    k_dot2<<<nb, AR_NT, 0, st>>>(w, w, dim, part, nullptr, S);
    k_ar_start<<<1, AR_NT, 0, st>>>(part, nb, S);
    k_ar_scale<<<nb, AR_NT, 0, st>>>(w, V, q, dim, S);
    HM_CUDA(cudaGetLastError());
    for (int j = 0; j < steps; ++j) {
        double *hcol = H + (size_t)j * (steps + 1);
        // w = H v_j from its binary64 copy q (a stopped run still launches the product;
        // its result is not used)
        HM_TRY(matvec_dev(b, bp, q, w, HM_F64, 1, st));
        // classical Gram-Schmidt, twice: h = V^T w, w -= V h, H[:, j] += h
        for (int pass = 0; pass < 2; ++pass) {
            k_mdot<<<L.nt, AR_NT, 0, st>>>(V, L.ldv, j + 1, w, dim, part, L.ps, S);
            k_mdot_fin<<<j + 1, AR_NT, 0, st>>>(part, L.nt, L.ps, h, hcol, S);
            k_gs_sub<<<nb, AR_NT, 0, st>>>(V, L.ldv, j + 1, h, w, dim, S);
        }
        k_dot2<<<nb, AR_NT, 0, st>>>(w, w, dim, part, nullptr, S);
        k_ar_beta<<<1, AR_NT, 0, st>>>(part, nb, hcol, j, S);
        k_ar_scale<<<nb, AR_NT, 0, st>>>(w, V + (size_t)(j + 1) * L.ldv, q, dim, S);
        HM_CUDA(cudaGetLastError());
    }
    ArState hs{};
    HM_CUDA(cudaMemcpyAsync(&hs, S, sizeof hs, cudaMemcpyDeviceToHost, st));
    std::vector<double> Hh((size_t)(steps + 1) * steps);
    HM_CUDA(cudaMemcpyAsync(Hh.data(), H, Hh.size() * 8, cudaMemcpyDeviceToHost, st));
    HM_CUDA(cudaStreamSynchronize(st));
    if (hs.status < 0) return fail(hs.status, "Arnoldi start vector has zero norm");
    const int m = hs.steps;
    *steps_done = m;
    if (hess) std::copy(Hh.begin(), Hh.end(), hess);
    if (n_ritz > 0) {
        // Ritz values: eigenvalues of the symmetric part of the leading m x m block of H
        std::vector<double> a((size_t)m * m), ev;
        for (int r = 0; r < m; ++r)
            for (int c = 0; c < m; ++c)
                a[(size_t)r * m + c] = 0.5 * (Hh[(size_t)c * (steps + 1) + r] + Hh[(size_t)r * (steps + 1) + c]);
        jacobi_eigenvalues(a, m, ev);
        for (int i = 0; i < n_ritz; ++i) ritz[i] = i < m ? ev[i] : NAN;
    }
    return hs.done && m < steps ? HM_BREAKDOWN : HM_OK;
}

int sym_eigenvalues(int n, const double *a, double *ev) {
    if (!a || !ev || n < 1 || n > 4096) return fail(HM_EINVAL, "sym_eigenvalues: NULL or n outside 1..4096");
    std::vector<double> s((size_t)n * n), w;
    for (int r = 0; r < n; ++r)
        for (int c = 0; c < n; ++c) s[(size_t)r * n + c] = 0.5 * (a[(size_t)r * n + c] + a[(size_t)c * n + r]);
    jacobi_eigenvalues(s, n, w);
    std::copy(w.begin(), w.end(), ev);
    return HM_OK;
}

int projection_workspace(const hm_basis *b, int steps, size_t *bytes) {
    if (!b || !bytes) return fail(HM_EINVAL, "NULL argument");
    if (steps < 1 || steps > 10000000) return fail(HM_EINVAL, "steps must be in 1..10^7");
    const uint64_t dim = b->view.dim;
    const int nb = grid_blocks(dim, AR_NT);
    *bytes = 2 * al256(dim * 8) + 2 * al256((size_t)nb * 8) + al256(sizeof(PrState)) + al256((size_t)steps * 8);
    return HM_OK;
}

int projection_run(const hm_basis *b, int n_bonds, const int32_t *u, const int32_t *v, const double *J,
                   const void *v0, uint64_t seed, int steps, double sigma, void *work, size_t work_bytes,
                   double *energies, double *psi_out, void *stream) {
    if (!b || !energies) return fail(HM_EINVAL, "NULL argument");
    if (b->parity) return fail(HM_EINVAL, "projection_run: not available on a spin-flip basis");
    if (!std::isfinite(sigma)) return fail(HM_EINVAL, "sigma must be finite");
    size_t need = 0;
    HM_TRY(projection_workspace(b, steps, &need));
    if (!work || work_bytes < need || ((uintptr_t)work & 255))
        return fail(HM_EWORKSPACE, "workspace must be >= %zu bytes, 256-byte aligned", need);
    BondParams bp;
    HM_TRY(make_bonds(b, n_bonds, u, v, J, &bp));
    if (sigma == 0.0) {             // default: sum_b |J_b| s (s + 1), a bound on |E| of H
        const double s = b->view.S2 / 2.0;
        for (int t = 0; t < n_bonds; ++t) sigma += std::fabs(J[t]) * s * (s + 1.0);
    }
    const uint64_t dim = b->view.dim;
    const int nb = grid_blocks(dim, AR_NT);
    unsigned char *W = (unsigned char *)work;
    size_t o = 0;
    double *psi = (double *)(W + o); o += al256(dim * 8);
    double *y = (double *)(W + o); o += al256(dim * 8);
    double *p1 = (double *)(W + o); o += al256((size_t)nb * 8);
    double *p2 = (double *)(W + o); o += al256((size_t)nb * 8);
    PrState *S = (PrState *)(W + o); o += al256(sizeof(PrState));
    double *E = (double *)(W + o);
    cudaStream_t st = as_stream(stream);
    // psi_0 = v0 / |v0| (the seeded uniform vector when v0 is NULL)
    if (v0) HM_CUDA(cudaMemcpyAsync(y, v0, dim * 8, cudaMemcpyDeviceToDevice, st));
    else HM_TRY(start_vector_dev(dim, seed, 0, y, HM_F64, st));
    k_dot2<<<nb, AR_NT, 0, st>>>(y, y, dim, p1, nullptr, nullptr);
    k_pr_start<<<1, AR_NT, 0, st>>>(p1, nb, S);
    k_pr_scale<<<nb, AR_NT, 0, st>>>(y, psi, dim, S);
    HM_CUDA(cudaGetLastError());
    // psi_{k+1} = (sigma - H) psi_k / |(sigma - H) psi_k|, E_k = psi_k . H psi_k
    for (int k = 0; k < steps; ++k) {
        HM_TRY(matvec_dev(b, bp, psi, y, HM_F64, 1, st));
        k_dot2<<<nb, AR_NT, 0, st>>>(psi, y, dim, p1, p2, nullptr);
        k_pr_fin<<<1, AR_NT, 0, st>>>(p1, p2, nb, sigma, E + k, S);
        k_pr_update<<<nb, AR_NT, 0, st>>>(psi, y, dim, sigma, S);
        HM_CUDA(cudaGetLastError());
    }
    PrState hs{};
    HM_CUDA(cudaMemcpyAsync(&hs, S, sizeof hs, cudaMemcpyDeviceToHost, st));
    HM_CUDA(cudaMemcpyAsync(energies, E, (size_t)steps * 8, cudaMemcpyDeviceToHost, st));
    if (psi_out) HM_CUDA(cudaMemcpyAsync(psi_out, psi, dim * 8, cudaMemcpyDeviceToDevice, st));
    HM_CUDA(cudaStreamSynchronize(st));
    if (hs.status < 0) return fail(hs.status, "projection start vector has zero norm");
    return HM_OK;
}

}  // extern "C"
