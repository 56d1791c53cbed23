// lanczos.cu -- the Lanczos recurrence around the row matvec, the tridiagonal
// eigensolvers on the device, lanczos_run (one CUDA graph) and e0_grad.
#include <algorithm>
#include <cmath>
#include <cstdio>
#include <cstring>
#include <new>

#include "blk.cuh"
#include "ef64.cuh"
#include "hm_row.cuh"
#include "s1blk.cuh"

namespace hm {

int blk_lz_plan(hm_basis *b, const BondParams &bp, int dtype, BlkParams *P, int *blocks);
int blk_lz_jit(const BlkParams &P, int dtype, const BondParams &bp, const void **kern, int *blocks, int split = 0);
int blk_lz_split(hm_basis *b, const BondParams &bp, const BlkParams &P, int dtype, BlkParams *PA, BlkParams *PB,
                 const void **kA, const void **kB, int *blkA, int *blkB);
int blk_target_table(hm_basis *b, BlkParams *P, int esize);
int blk_K(const hm_basis *b);   // blk.cu: split position of the block path
int blk_lz64_launch(const BlkParams &P, const long long *Xc, unsigned long long *Y, LzScalars *S, int pc,
                    double *part, int blocks, cudaStream_t st, const void *jit);
int blk_lz32_launch(const BlkParams &P, const float *qc, float *qp, LzScalars *S, double *part, int blocks,
                    cudaStream_t st, const void *jit);

int matvec_dev(const hm_basis *b, const BondParams &bp, const void *x, void *y, int dtype,
               int nvec, cudaStream_t st);
int bond_corr_dev(const hm_basis *b, const BondParams &bp, const void *g, const void *x,
                  double *out, int dtype, void *work, size_t work_bytes, double sign,
                  const double *div, cudaStream_t st);
size_t bond_corr_bytes(const hm_basis *b, int n_bonds);
int start_vector_dev(uint64_t n, uint64_t seed, int kind, void *x, int dtype, cudaStream_t st);

// breakdown: beta_j <= LZ_TOL * max(|alpha|, beta).  FP64 vectors are updated in double-float
// arithmetic (about 2^-48 unit roundoff, not binary64's 2^-53), so a beta that vanishes in
// exact arithmetic comes out near 1e-12 of the scale; the threshold sits well above that floor.
constexpr double LZ_TOL = 1e-10;
constexpr double LZ_TOL32 = 1e-5;    // FP32 vectors: above their rounding floor
constexpr int NT = 256;

// workspace carve-up (all segments 256-byte aligned)
struct LzLayout {
    size_t buf[2], part, sc, alpha, beta, ritz, psi, coef, res, gout, tri, bpart, total;
    size_t ybuf, xs[2];     // FP64 block path: y = H q and the fixed-point copies of q
    size_t qqp;             // FP64 block path: partials of q_cur . q_prev (update kernel)
    size_t hpart;           // s = 1/2 block path: per-block partial sums, 2 x 2^hpart_H doubles
    int hpart_H;
    size_t s1part;          // s = 1 block path: one partial sum per block, s1n of them
    size_t mv;              // momentum basis: y = H q from the momentum product
    uint64_t s1n;
    bool shadow;
};

static size_t al256(size_t x) { return (x + 255) & ~(size_t)255; }

static LzLayout lz_layout(const hm_basis *b, int dtype, int max_steps, bool grad, int nb) {
    LzLayout L{};
    const uint64_t dim = b->view.dim;
    const size_t es = dtype == HM_F64 ? 8 : 4;
    const int nblk = grid_blocks(dim, NT);
    size_t o = 0;
    L.buf[0] = o; o += al256(dim * es);
    L.buf[1] = o; o += al256(dim * es);
    const size_t npart = std::max<size_t>((size_t)nblk, (size_t)sm_count() * 8);
    L.part = o; o += al256(npart * 2 * sizeof(double));
    // the block paths of FP64 runs (s = 1/2, s = 1) need y and two fixed-point copies; a
    // momentum basis takes neither block path but needs y = H q
    const bool mom = b->mom_k >= 0;
    const uint64_t s1n = mom ? 0 : s1_block_count(b);
    L.shadow = !mom && dtype == HM_F64 && !b->view.idx64 &&
               ((b->view.S2 == 1 && b->view.N >= 10 && b->view.N <= 32) || (b->view.S2 == 2 && s1n > 0));
    if (mom) { L.mv = o; o += al256(dim * es); }
    if (L.shadow) {
        L.ybuf = o; o += al256(dim * 8);
        L.xs[0] = o; o += al256(dim * 8);
        L.xs[1] = o; o += al256(dim * 8);
        L.qqp = o; o += al256(npart * sizeof(double));
    }
    // per-block partials of the s = 1/2 block path (split K = min(15, N - 2): H <= 17)
    if (!mom && b->view.S2 == 1 && b->view.N >= 10 && b->view.N <= 32 && !b->view.idx64) {
        const int H = b->view.N - blk_K(b);
        L.hpart_H = H;
        L.hpart = o; o += al256(((size_t)2 << H) * sizeof(double));
    }
    // per-block partials of the s = 1 block path
    if ((L.s1n = s1n) > 0) { L.s1part = o; o += al256(L.s1n * sizeof(double)); }
    L.sc = o; o += al256(sizeof(LzScalars));
    L.alpha = o; o += al256((size_t)max_steps * 8);
    L.beta = o; o += al256((size_t)max_steps * 8);
    L.ritz = o; o += al256(64 * 8);
    if (grad) {
        L.psi = o; o += al256(dim * 8);
        L.coef = o; o += al256((size_t)max_steps * 8);
        L.res = o; o += al256((size_t)max_steps * 8);
        L.gout = o; o += al256((size_t)(nb > 0 ? nb : 1) * 8);
        // per-length convergence scratch: max_steps x (5 * max_steps) doubles
        L.tri = o; o += al256((size_t)max_steps * (5 * (size_t)max_steps + 4) * 8);
        L.bpart = o; o += al256(bond_corr_bytes(b, nb));
    }
    L.total = o;
    return L;
}

}  // namespace hm

struct hm_lanczos {
    const hm_basis *basis;
    hm::BondParams bp;
    hm::BlkParams blk;      // s = 1/2 block path (use_blk)
    int use_blk, blk_blocks;
    const void *jit;        // block product specialised to the bonds (jit.cu), or nullptr
    // split FP64 product (blk_lz_split): blk / jit / blk_blocks are pass 1, these pass 2
    int split, blk_blocks2;
    hm::BlkParams blk2;
    const void *jit2;
    int run;                // rows per thread run of the general product (row_runs)
    int use_s1;             // s = 1 block path (s1blk.cu)
    int use_mom;            // momentum basis: product k_mom_matvec, then the epilogue kernel
    hm::S1Plan s1;
    int dtype, max_steps, host_j, next_phase;
    unsigned char *work;
    hm::LzLayout L;
    hm::LzScalars *sc;
    double *alpha, *beta, *part, *psi, *coef;
    double *hpart;          // per-block partials of the block path (entries of absent blocks stay 0)
    double *qqp;            // partials of q_cur . q_prev (FP64 block path, from the update)
};

namespace hm {

// ---------------------------------------------------------------------------------------
// kernels
// ---------------------------------------------------------------------------------------
// part[blk] = sum q^2 (double-float per thread); *emax = max exponent field (if given)
template <class T>
__global__ void __launch_bounds__(NT) k_sumsq(const T *__restrict__ q, uint64_t n, double *__restrict__ part,
                                               int *emax) {
    __shared__ double red[NT / 32];
    ef::df s{0.0f, 0.0f};
    double sd = 0.0;
    int em = 0;
    for (uint64_t r = blockIdx.x * (uint64_t)NT + threadIdx.x; r < n; r += (uint64_t)gridDim.x * NT) {
        if constexpr (sizeof(T) == 8) {
            const unsigned long long b = ((const unsigned long long *)q)[r];
            em = max(em, (int)((b >> 52) & 0x7FF));
            sd += q[r] * q[r];   // start vector only: once per run
        } else {
            s = ef::df_add(s, ef::two_prod(q[r], q[r]));
        }
    }
    double tot = block_sum<NT>(sd + (double)s.hi + (double)s.lo, red);
    if (threadIdx.x == 0) part[blockIdx.x] = tot;
    if (emax) {
        for (int o = 16; o > 0; o >>= 1) em = max(em, __shfl_down_sync(0xffffffffu, em, o));
        if ((threadIdx.x & 31) == 0) atomicMax(emax, em);
    }
}

// scalars were zeroed (emax[0] filled by k_sumsq) before this runs
__global__ void k_lz_start(LzScalars *S, const double *__restrict__ part, int nblk) {
    __shared__ double red[NT / 32];
    double s = 0.0;
    for (int k = threadIdx.x; k < nblk; k += NT) s += part[k];
    s = block_sum<NT>(s, red);
    if (threadIdx.x == 0) {
        S->sigma_cur = 1.0 / sqrt(s);
        S->done = (s > 0.0) ? 0 : 1;
        S->status = (s > 0.0) ? HM_OK : HM_EINVAL;
    }
}

// u = sigma_cur * H q_cur - beta_prev * sigma_prev * q_prev, written over q_prev;
// part[blk] = sum (sigma_cur q_cur) . u
template <class I, class T, class Acc>
__global__ void __launch_bounds__(NT)
k_lz_matvec(SectorView sv, BondParams bp, const T *__restrict__ qc, T *__restrict__ qp,
            const LzScalars *__restrict__ S, double *__restrict__ part, int run) {
    if (S->done) return;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    __shared__ double red[NT / 32];
    const double *pdn, *pup;
    const I *cd = stage_tables<I>(sv, bp, smem_raw, &pdn, &pup);
    I *const px = row_px_base<I>(sv, smem_raw);
    Codec<I> c{cd, sv.N, sv.S2, sv.A, sv.bits, sv.cd_w, sv.cd_rowlen};
    const double sc = S->sigma_cur, bp_ = S->beta_prev * S->sigma_prev;
    const float scf = (float)sc, bpf = (float)bp_;
    double dot = 0.0;
    ef::df dotf{0.0f, 0.0f};
    row_runs(c, sv.dim, px, run, [&](uint64_t r, uint64_t w) {
        const I i = (I)r;
        Acc acc[1], dg;
        row_apply<I, T, Acc, 1>(c, bp, pdn, pup, i, w, qc, 1, 0, acc, &dg, px);
        const Acc hv = dg * (Acc)qc[r] + acc[0];
        if constexpr (sizeof(T) == 8) {
            const T u = (T)(sc * (double)hv - bp_ * (double)qp[r]);
            qp[r] = u;
            dot += (sc * (double)qc[r]) * (double)u;
        } else {
            const float u = scf * (float)hv - bpf * (float)qp[r];
            qp[r] = (T)u;
            dotf = ef::df_add(dotf, ef::two_prod(scf * (float)qc[r], u));
        }
    });
    dot = block_sum<NT>(dot + (double)dotf.hi + (double)dotf.lo, red);
    if (threadIdx.x == 0) part[blockIdx.x] = dot;
}

// the epilogue of k_lz_matvec for a product formed by another kernel (momentum basis):
// u = sigma_cur y - beta_prev sigma_prev q_prev over q_prev, part[blk] = sum (sigma_cur q_cur) . u
template <class T>
__global__ void __launch_bounds__(NT) k_lz_mv_epi(const T *__restrict__ y, const T *__restrict__ qc,
                                                   T *__restrict__ qp, uint64_t n, const LzScalars *__restrict__ S,
                                                   double *__restrict__ part) {
    if (S->done) return;
    __shared__ double red[NT / 32];
    const double sc = S->sigma_cur, bp_ = S->beta_prev * S->sigma_prev;
    const float scf = (float)sc, bpf = (float)bp_;
    double dot = 0.0;
    ef::df dotf{0.0f, 0.0f};
    for (uint64_t r = (uint64_t)blockIdx.x * NT + threadIdx.x; r < n; r += (uint64_t)gridDim.x * NT) {
        if constexpr (sizeof(T) == 8) {
            const T u = (T)(sc * (double)y[r] - bp_ * (double)qp[r]);
            qp[r] = u;
            dot += (sc * (double)qc[r]) * (double)u;
        } else {
            const float u = scf * (float)y[r] - bpf * (float)qp[r];
            qp[r] = (T)u;
            dotf = ef::df_add(dotf, ef::two_prod(scf * (float)qc[r], u));
        }
    }
    dot = block_sum<NT>(dot + (double)dotf.hi + (double)dotf.lo, red);
    if (threadIdx.x == 0) part[blockIdx.x] = dot;
}

__global__ void k_lz_alpha(LzScalars *S, const double *__restrict__ part, int nblk, double *alpha,
                           int pprev) {
    if (S->done) return;
    __shared__ double red[NT / 32];
    double s = 0.0;
    for (int k = threadIdx.x; k < nblk; k += NT) s += part[k];
    s = block_sum<NT>(s, red);
    if (threadIdx.x == 0) {
        alpha[S->j] = s;
        S->scale = fmax(S->scale, fabs(s));
        S->emax[pprev] = 0;          // filled again by the update kernel
    }
}

// w = u - alpha_j sigma_cur q_cur over q_prev; part = sum w^2; psi += coef_j v_j if PSI.
// FP64 in double-float arithmetic on the bit patterns (no FP64 instruction per row
// unless PSI: a run-time test of psi inside the loop would be predicated, not branched
// around, and the psi terms would cost binary64 instructions on every row);
// the largest exponent field of w goes to S->emax[pprev].
template <class T, bool PSI>
__global__ void __launch_bounds__(NT)
k_lz_update(const T *__restrict__ qc, T *__restrict__ qp, uint64_t n, LzScalars *S,
            const double *__restrict__ alpha, double *__restrict__ part, double *__restrict__ psi,
            const double *__restrict__ coef, int pprev) {
    if (S->done) return;
    __shared__ double red[NT / 32];
    const double as = alpha[S->j] * S->sigma_cur;
    const double cj = psi ? coef[S->j] * S->sigma_cur : 0.0;
    const int scale_q = S->emax[pprev ^ 1] - 1023;
    const ef::df as_s = [&] { const double v = ldexp(as, scale_q); const float h = (float)v; return ef::df{h, (float)(v - (double)h)}; }();
    const float asf = (float)as;
    ef::df s{0.0f, 0.0f};
    int em = 0;
    uint64_t r0 = 0;
    if constexpr (sizeof(T) == 4 && !PSI) {
        // FP32 without psi: four rows per 16-byte load (the buffers are 256-byte aligned), so
        // that each thread keeps more bytes in flight; the rows past the last multiple of
        // four go through the loop below
        const uint64_t n4 = n / 4;
        const float4 *qc4 = reinterpret_cast<const float4 *>(qc);
        float4 *qp4 = reinterpret_cast<float4 *>(qp);
        for (uint64_t r = blockIdx.x * (uint64_t)NT + threadIdx.x; r < n4; r += (uint64_t)gridDim.x * NT) {
            const float4 u = qp4[r], x = __ldcs(qc4 + r);
            float4 w;
            w.x = u.x - asf * x.x; w.y = u.y - asf * x.y;
            w.z = u.z - asf * x.z; w.w = u.w - asf * x.w;
            qp4[r] = w;
            s = ef::df_add(s, ef::two_prod(w.x, w.x));
            s = ef::df_add(s, ef::two_prod(w.y, w.y));
            s = ef::df_add(s, ef::two_prod(w.z, w.z));
            s = ef::df_add(s, ef::two_prod(w.w, w.w));
        }
        r0 = 4 * n4;
    }
    for (uint64_t r = r0 + blockIdx.x * (uint64_t)NT + threadIdx.x; r < n; r += (uint64_t)gridDim.x * NT) {
        if constexpr (sizeof(T) == 8) {
            const unsigned long long qb = ((const unsigned long long *)qc)[r];
            const unsigned long long ub = ((const unsigned long long *)qp)[r];
            const ef::df w = ef::df_add(ef::df_from_bits(ub, 0),
                                        ef::df_neg(ef::df_mul(as_s, ef::df_from_bits(qb, scale_q))));
            const unsigned long long wb = ef::bits_from_df(w, 0);
            ((unsigned long long *)qp)[r] = wb;
            em = max(em, (int)((wb >> 52) & 0x7FF));
            s = ef::df_add(s, ef::df_mul(w, w));
            if constexpr (PSI) psi[r] += cj * ef::u2d(qb);
        } else {
            const float w = qp[r] - asf * qc[r];
            qp[r] = w;
            s = ef::df_add(s, ef::two_prod(w, w));
            if constexpr (PSI) psi[r] += cj * (double)qc[r];
        }
    }
    const double tot = block_sum<NT>((double)s.hi + (double)s.lo, red);
    if (threadIdx.x == 0) part[blockIdx.x] = tot;
    if constexpr (sizeof(T) == 8) {
        for (int o = 16; o > 0; o >>= 1) em = max(em, __shfl_down_sync(0xffffffffu, em, o));
        if ((threadIdx.x & 31) == 0) atomicMax(&S->emax[pprev], em);
    }
}

// alpha_j = sigma^2 (q.Hq) - sigma gamma (q.q_prev): q.Hq from the per-block partials of
// the FP64 block product (exact integer dots of the fixed-point copy), q.q_prev from those
// of the update kernel that made q (double-float), zero at the start (the Paige form
// v.(Hv - beta v_prev))
__global__ void k_lz_alpha2(LzScalars *S, const double *__restrict__ part, int nblk, const double *__restrict__ qqp,
                            int nq, double *alpha, int pprev) {
    if (S->done) return;
    __shared__ double red[NT / 32];
    double s1 = 0.0, s2 = 0.0;
    for (int k = threadIdx.x; k < nblk; k += NT) s1 += part[k];
    for (int k = threadIdx.x; k < nq; k += NT) s2 += qqp[k];
    s1 = block_sum<NT>(s1, red);
    __syncthreads();
    s2 = block_sum<NT>(s2, red);
    if (threadIdx.x == 0) {
        const double sg = S->sigma_cur, gm = S->beta_prev * S->sigma_prev;
        const double a = sg * sg * s1 - sg * gm * s2;
        alpha[S->j] = a;
        S->scale = fmax(S->scale, fabs(a));
        S->emax_old = S->emax[pprev];
        S->emax[pprev] = 0;          // filled again by the update kernel
    }
}

// Resident CTAs per SM of the FP64 block path's update: 40 registers a thread (at 8 CTAs
// and 32 registers its double-float dots spill; N = 32 step 20.21 against 20.09 ms with the
// spills and 19.82 ms here).  The update and the reductions of its partials run on a grid
// of this many CTAs per SM (upd64_blocks).
constexpr int UPD64_CTAS = 6;
static int upd64_blocks(uint64_t dim) { return std::min(grid_blocks(dim, NT), sm_count() * UPD64_CTAS); }

// FP64 block path.  The Lanczos vectors are kept as double-float pairs (hi, lo floats,
// 8 bytes): the update computes in double-float, so a pair holds all it produces and
// needs no conversion to or from binary64.
// w = sigma y - alpha sigma q - gamma q_prev over q_prev (y: binary64 bits of H q);
// part = |w|^2; qqp = w . q (the stored new and current vectors, for the next alpha; both
// dots in double-float per thread, binary64 over the block); largest exponent of w, as a
// binary64 exponent field, to S->emax[pprev]; psi += coef_j q if PSI
template <bool PSI>
__global__ void __launch_bounds__(NT, UPD64_CTAS)
k_lz_update_y(const unsigned long long *__restrict__ Y, const float2 *__restrict__ qc, float2 *__restrict__ qp,
              uint64_t n, LzScalars *S, const double *__restrict__ alpha, double *__restrict__ part,
              double *__restrict__ qqp, double *__restrict__ psi, const double *__restrict__ coef, int pprev) {
    if (S->done) return;
    __shared__ double red[NT / 32];
    const double sg = S->sigma_cur, gm = S->beta_prev * S->sigma_prev, as = alpha[S->j] * sg;
    const double cj = psi ? coef[S->j] * sg : 0.0;
    auto todf = [](double v) { const float h = (float)v; return ef::df{h, (float)(v - (double)h)}; };
    const ef::df sg_d = todf(sg), as_d = todf(as), gm_d = todf(gm);
    ef::df s{0.0f, 0.0f}, dq{0.0f, 0.0f};
    uint32_t eh = 0;
    auto row = [&](unsigned long long yb, float2 q2, float2 p2) {
        const ef::df q = ef::df{q2.x, q2.y};
        const ef::df t1 = ef::df_mul(sg_d, ef::df_from_bits(yb, 0));
        const ef::df t2 = ef::df_mul(as_d, q);
        const ef::df t3 = ef::df_mul(gm_d, ef::df{p2.x, p2.y});
        const ef::df w = ef::df_add(t1, ef::df_neg(ef::df_add(t2, t3)));
        eh = max(eh, (ef::f2u(w.hi) >> 23) & 0xFFu);
        s = ef::df_add(s, ef::df_mul(w, w));
        dq = ef::df_add(dq, ef::df_mul(w, q));
        return make_float2(w.hi, w.lo);
    };
    const uint64_t stride = (uint64_t)gridDim.x * NT;
    uint64_t r0 = 0;
    if constexpr (!PSI) {
        // two rows per 16-byte access of each operand (the buffers are 256-byte aligned), so
        // that each thread keeps more bytes in flight; an odd last row goes through the loop
        // below
        const uint64_t n2 = n / 2;
        const ulonglong2 *Y2 = reinterpret_cast<const ulonglong2 *>(Y);
        const float4 *qc2 = reinterpret_cast<const float4 *>(qc);
        float4 *qp2 = reinterpret_cast<float4 *>(qp);
        for (uint64_t r = blockIdx.x * (uint64_t)NT + threadIdx.x; r < n2; r += stride) {
            const ulonglong2 yb = __ldcs(Y2 + r);
            const float4 q4 = __ldcs(qc2 + r), p4 = qp2[r];
            const float2 w0 = row(yb.x, make_float2(q4.x, q4.y), make_float2(p4.x, p4.y));
            const float2 w1 = row(yb.y, make_float2(q4.z, q4.w), make_float2(p4.z, p4.w));
            qp2[r] = make_float4(w0.x, w0.y, w1.x, w1.y);
        }
        r0 = 2 * n2;
    }
    for (uint64_t r = r0 + blockIdx.x * (uint64_t)NT + threadIdx.x; r < n; r += stride) {
        const float2 q2 = __ldcs(qc + r);
        qp[r] = row(__ldcs(Y + r), q2, qp[r]);
        if constexpr (PSI) psi[r] += cj * ((double)q2.x + (double)q2.y);
    }
    const double tot = block_sum<NT>((double)s.hi + (double)s.lo, red);
    if (threadIdx.x == 0) part[blockIdx.x] = tot;
    __syncthreads();
    const double tq = block_sum<NT>((double)dq.hi + (double)dq.lo, red);
    if (threadIdx.x == 0) qqp[blockIdx.x] = tq;
    for (int o = 16; o > 0; o >>= 1) eh = max(eh, __shfl_down_sync(0xffffffffu, eh, o));
    // |hi| < 2^(eh - 126): the binary64 field eh - 127 + 1023 bounds hi, and hi + lo up
    // to a factor 1 + 2^-24 (the fixed-point copy then stays within 2^53 + 2^29 units)
    if ((threadIdx.x & 31) == 0 && eh) atomicMax(&S->emax[pprev], (int)eh - 127 + 1023);
}

// start vector of the FP64 block path, one pass: its fixed-point copy X (unit from its
// largest exponent field, S->emax[0]) and the binary64 values turned into double-float
// pairs in place (integer conversion, no FP64 instruction); there is no vector before it,
// so its q.q_prev partials are zero
__global__ void __launch_bounds__(NT) k_fix_start(unsigned long long *__restrict__ b, long long *__restrict__ X,
                                                  uint64_t n, const LzScalars *S, double *__restrict__ qqp) {
    const int E = S->emax[0];
    for (uint64_t r = blockIdx.x * (uint64_t)NT + threadIdx.x; r < n; r += (uint64_t)gridDim.x * NT) {
        const unsigned long long v = b[r];
        __stcs(X + r, (long long)ef::fix_from_bits(v, E));
        const ef::df d = ef::df_from_bits(v, 0);
        ((float2 *)b)[r] = make_float2(d.hi, d.lo);
    }
    if (threadIdx.x == 0) qqp[blockIdx.x] = 0.0;
}

// fixed-point copy X of the new vector w (double-float pairs), unit from its largest
// exponent (the dot with the current vector for the next alpha comes from the update)
__global__ void __launch_bounds__(NT, 2048 / NT)
k_fixd(const float2 *__restrict__ w, long long *__restrict__ X, uint64_t n, const LzScalars *S, int slot) {
    if (S->done) return;
    const int E = S->emax[slot];
    const uint64_t stride = (uint64_t)gridDim.x * NT;
    // two rows per 16-byte access (256-byte aligned buffers); an odd last row after
    const uint64_t n2 = n / 2;
    const float4 *w2 = reinterpret_cast<const float4 *>(w);
    longlong2 *X2 = reinterpret_cast<longlong2 *>(X);
    for (uint64_t r = blockIdx.x * (uint64_t)NT + threadIdx.x; r < n2; r += stride) {
        const float4 v = __ldcs(w2 + r);
        longlong2 x;
        x.x = (long long)ef::fix_from_df(ef::df{v.x, v.y}, E, 0);
        x.y = (long long)ef::fix_from_df(ef::df{v.z, v.w}, E, 0);
        __stcs(X2 + r, x);
    }
    for (uint64_t r = 2 * n2 + blockIdx.x * (uint64_t)NT + threadIdx.x; r < n; r += stride)
        __stcs(X + r, (long long)ef::fix_from_df(ef::df{w[r].x, w[r].y}, E, 0));
}

__global__ void k_lz_beta(LzScalars *S, const double *__restrict__ part, int nblk, double *beta, double tol) {
    if (S->done) return;
    __shared__ double red[NT / 32];
    double s = 0.0;
    for (int k = threadIdx.x; k < nblk; k += NT) s += part[k];
    s = block_sum<NT>(s, red);
    if (threadIdx.x == 0) {
        const double b = sqrt(s);
        beta[S->j] = b;
        S->j += 1;
        if (b <= tol * S->scale) {
            S->done = 1;
            S->status = HM_BREAKDOWN;
        } else {
            S->scale = fmax(S->scale, b);
            S->sigma_prev = S->sigma_cur;
            S->sigma_cur = 1.0 / b;
            S->beta_prev = b;
        }
    }
}

// ---- tridiagonal T (diagonal al[0..m), off-diagonal be[0..m-1)) ------------------------

__device__ int sturm_count(int m, const double *al, const double *be, double x, double pivmin) {
    int c = 0;
    double q = al[0] - x;
    if (fabs(q) < pivmin) q = -pivmin;
    if (q < 0) ++c;
    for (int i = 1; i < m; ++i) {
        q = (al[i] - x) - be[i - 1] * be[i - 1] / q;
        if (fabs(q) < pivmin) q = -pivmin;
        if (q < 0) ++c;
    }
    return c;
}

// e-th lowest eigenvalue (1-based) by bisection of the Sturm count on the Gershgorin
// interval, until the midpoint no longer moves
__device__ double tri_eig(int m, const double *al, const double *be, int e) {
    double lo = 1e308, hi = -1e308, bmax = 0.0;
    for (int i = 0; i < m; ++i) {
        double r = (i > 0 ? fabs(be[i - 1]) : 0.0) + (i < m - 1 ? fabs(be[i]) : 0.0);
        lo = fmin(lo, al[i] - r);
        hi = fmax(hi, al[i] + r);
        if (i < m - 1) bmax = fmax(bmax, fabs(be[i]));
    }
    const double pivmin = 2.2250738585072014e-308 * fmax(1.0, bmax * bmax);
    const double pad = 2.0 * 2.220446049250313e-16 * fmax(fabs(lo), fabs(hi)) + pivmin;
    double a = lo - pad, c = hi + pad;
    for (int it = 0; it < 400; ++it) {
        double mid = 0.5 * (a + c);
        if (mid <= a || mid >= c) break;
        if (sturm_count(m, al, be, mid, pivmin) >= e) c = mid; else a = mid;
    }
    return 0.5 * (a + c);
}

// eigenvector of T for eigenvalue th by inverse iteration: three solves of
// (T - th I) z = b with Gaussian elimination and partial pivoting (one extra
// super-diagonal of fill-in); z normalised, returned in z[0..m)
__device__ void tri_vec(int m, const double *al, const double *be, double th, double *z,
                        double *d, double *du, double *du2, double *dl) {
    if (m == 1) { z[0] = 1.0; return; }
    double tnorm = 0.0;
    for (int i = 0; i < m; ++i) tnorm = fmax(tnorm, fabs(al[i]) + (i > 0 ? fabs(be[i - 1]) : 0.0) + (i < m - 1 ? fabs(be[i]) : 0.0));
    const double tiny = fmax(tnorm, 1e-300) * 2.220446049250313e-16;
    for (int i = 0; i < m; ++i) z[i] = 1.0 / sqrt((double)m) * (1.0 + 1e-3 * (double)(i % 7));
    for (int it = 0; it < 3; ++it) {
        for (int i = 0; i < m; ++i) d[i] = al[i] - th;
        for (int i = 0; i < m - 1; ++i) { du[i] = be[i]; dl[i] = be[i]; }
        for (int i = 0; i < m; ++i) du2[i] = 0.0;
        double *b = z;
        for (int i = 0; i < m - 1; ++i) {
            if (fabs(d[i]) >= fabs(dl[i])) {
                if (d[i] == 0.0) d[i] = tiny;
                const double f = dl[i] / d[i];
                d[i + 1] -= f * du[i];
                b[i + 1] -= f * b[i];
            } else {
                const double f = d[i] / dl[i];
                d[i] = dl[i];
                const double t = d[i + 1];
                d[i + 1] = du[i] - f * t;
                du[i] = t;
                if (i < m - 2) {
                    du2[i] = du[i + 1];
                    du[i + 1] = -f * du[i + 1];
                }
                const double tb = b[i];
                b[i] = b[i + 1];
                b[i + 1] = tb - f * b[i + 1];
            }
        }
        if (d[m - 1] == 0.0) d[m - 1] = tiny;
        b[m - 1] = b[m - 1] / d[m - 1];
        b[m - 2] = (b[m - 2] - du[m - 2] * b[m - 1]) / d[m - 2];
        for (int i = m - 3; i >= 0; --i) b[i] = (b[i] - du[i] * b[i + 1] - du2[i] * b[i + 2]) / d[i];
        double nn = 0.0;
        for (int i = 0; i < m; ++i) nn += b[i] * b[i];
        nn = 1.0 / sqrt(nn);
        for (int i = 0; i < m; ++i) b[i] *= nn;
    }
}

__global__ void k_ritz(const LzScalars *S, const double *alpha, const double *beta, int n_ritz, double *ritz) {
    const int e = blockIdx.x * blockDim.x + threadIdx.x;
    const int m = S->j;
    if (e >= n_ritz) return;
    ritz[e] = (m >= 1 && e < m) ? tri_eig(m, alpha, beta, e + 1) : __longlong_as_double(0x7ff8000000000000ll);
}

// Convergence of the lowest Ritz pair of every leading T_k (k = 1..m): thread k computes
// theta_1(T_k) and the last component s_k of its eigenvector; the residual norm of the
// Ritz pair is beta_k |s_k|.  res[k-1] = beta_k |s_k| / max(1, |theta|).
__global__ void k_conv_scan(const LzScalars *S, const double *alpha, const double *beta,
                            double *scratch, int max_steps, double *res) {
    const int k = blockIdx.x * blockDim.x + threadIdx.x + 1;
    const int m = S->j;
    if (k > m) return;
    double *z = scratch + (size_t)(k - 1) * (5 * (size_t)max_steps + 4);
    double *d = z + max_steps, *du = d + max_steps, *du2 = du + max_steps, *dl = du2 + max_steps;
    const double th = tri_eig(k, alpha, beta, 1);
    tri_vec(k, alpha, beta, th, z, d, du, du2, dl);
    res[k - 1] = beta[k - 1] * fabs(z[k - 1]) / fmax(1.0, fabs(th));
}

// picks the shortest converged Krylov length (res <= tol), or m; computes the lowest
// eigenvector of T_mconv into coef, and e0 / e1 into ritz[0], ritz[1]
__global__ void k_pick_and_vec(LzScalars *S, const double *alpha, const double *beta,
                               double *scratch, int max_steps, const double *res, double tol,
                               double *coef, double *ritz) {
    if (threadIdx.x != 0 || blockIdx.x != 0) return;
    const int m = S->j;
    int mc = m;
    for (int k = 1; k <= m; ++k)
        if (res[k - 1] <= tol) { mc = k; break; }
    S->mconv = mc;
    double *d = scratch, *du = d + max_steps, *du2 = du + max_steps, *dl = du2 + max_steps;
    const double th = tri_eig(mc, alpha, beta, 1);
    ritz[0] = th;
    ritz[1] = mc >= 2 ? tri_eig(mc, alpha, beta, 2) : __longlong_as_double(0x7ff0000000000000ll);
    tri_vec(mc, alpha, beta, th, coef, d, du, du2, dl);
    for (int k = mc; k < max_steps; ++k) coef[k] = 0.0;
}

__global__ void k_scale(double *__restrict__ v, uint64_t n, const LzScalars *S) {
    const double f = 1.0 / sqrt(S->nrm2);
    for (uint64_t r = blockIdx.x * (uint64_t)NT + threadIdx.x; r < n; r += (uint64_t)gridDim.x * NT) v[r] *= f;
}

__global__ void k_store_nrm2(LzScalars *S, const double *__restrict__ part, int nblk) {
    __shared__ double red[NT / 32];
    double s = 0.0;
    for (int k = threadIdx.x; k < nblk; k += NT) s += part[k];
    s = block_sum<NT>(s, red);
    if (threadIdx.x == 0) S->nrm2 = s;
}

// ---------------------------------------------------------------------------------------
// host side
// ---------------------------------------------------------------------------------------
template <class I, class T, class Acc>
static int enqueue_phase_t(hm_lanczos *R, int parity, int phase, cudaStream_t st) {
    const SectorView &sv = R->basis->view;
    T *b0 = (T *)(R->work + R->L.buf[0]);
    T *b1 = (T *)(R->work + R->L.buf[1]);
    T *qc = parity ? b1 : b0;
    T *qp = parity ? b0 : b1;
    const int nblk = grid_blocks(sv.dim, NT);
    const int pprev = parity ^ 1;   // buffer of q_prev, receives u then w
    const bool b64 = (R->use_blk || R->use_s1) && R->dtype == HM_F64;
    const int nblk64 = upd64_blocks(sv.dim);   // grid of the FP64 block path's update kernels
    long long *xs[2] = {R->L.shadow ? (long long *)(R->work + R->L.xs[0]) : nullptr,
                        R->L.shadow ? (long long *)(R->work + R->L.xs[1]) : nullptr};
    unsigned long long *Y = R->L.shadow ? (unsigned long long *)(R->work + R->L.ybuf) : nullptr;
    if (phase == 0) {
        if (R->use_mom) {
            T *y = (T *)(R->work + R->L.mv);
            HM_TRY(matvec_dev(R->basis, R->bp, qc, y, R->dtype, 1, st));
            k_lz_mv_epi<T><<<nblk, NT, 0, st>>>(y, qc, qp, sv.dim, R->sc, R->part);
            k_lz_alpha<<<1, NT, 0, st>>>(R->sc, R->part, nblk, R->alpha, pprev);
        } else if (b64 && R->use_s1) {
            double *s1part = (double *)(R->work + R->L.s1part);
            HM_TRY(s1_lz64(R->s1, xs[parity], Y, R->sc, parity, s1part, st));
            k_lz_alpha2<<<1, NT, 0, st>>>(R->sc, s1part, R->s1.nblocks, R->qqp, nblk64, R->alpha, pprev);
        } else if (b64) {
            HM_TRY(blk_lz64_launch(R->blk, xs[parity], Y, R->sc, parity, R->hpart, R->blk_blocks, st, R->jit));
            if (R->split)
                HM_TRY(blk_lz64_launch(R->blk2, xs[parity], Y, R->sc, parity, R->hpart, R->blk_blocks2, st, R->jit2));
            k_lz_alpha2<<<1, NT, 0, st>>>(R->sc, R->hpart, 1 << R->blk.H, R->qqp, nblk64, R->alpha, pprev);
        } else if (R->use_blk) {
            HM_TRY(blk_lz32_launch(R->blk, (const float *)qc, (float *)qp, R->sc, R->hpart, R->blk_blocks, st, R->jit));
            k_lz_alpha<<<1, NT, 0, st>>>(R->sc, R->hpart, 1 << R->blk.H, R->alpha, pprev);
        } else if (R->use_s1) {
            double *s1part = (double *)(R->work + R->L.s1part);
            HM_TRY(s1_lz32(R->s1, (const float *)qc, (float *)qp, R->sc, s1part, st));
            k_lz_alpha<<<1, NT, 0, st>>>(R->sc, s1part, R->s1.nblocks, R->alpha, pprev);
        } else {
            const size_t sm = row_smem_bytes<I>(sv);
            k_lz_matvec<I, T, Acc><<<nblk, NT, sm, st>>>(sv, R->bp, qc, qp, R->sc, R->part, R->run);
            k_lz_alpha<<<1, NT, 0, st>>>(R->sc, R->part, nblk, R->alpha, pprev);
        }
    } else if (b64) {
        if (R->psi)
            k_lz_update_y<true><<<nblk64, NT, 0, st>>>(Y, (const float2 *)qc, (float2 *)qp, sv.dim, R->sc, R->alpha,
                                                       R->part, R->qqp, R->psi, R->coef, pprev);
        else
            k_lz_update_y<false><<<nblk64, NT, 0, st>>>(Y, (const float2 *)qc, (float2 *)qp, sv.dim, R->sc,
                                                        R->alpha, R->part, R->qqp, nullptr, R->coef, pprev);
        k_lz_beta<<<1, NT, 0, st>>>(R->sc, R->part, nblk64, R->beta, R->dtype == HM_F64 ? LZ_TOL : LZ_TOL32);
        k_fixd<<<nblk, NT, 0, st>>>((const float2 *)qp, xs[pprev], sv.dim, R->sc, pprev);
    } else {
        if (R->psi)
            k_lz_update<T, true><<<nblk, NT, 0, st>>>(qc, qp, sv.dim, R->sc, R->alpha, R->part, R->psi, R->coef, pprev);
        else
            k_lz_update<T, false><<<nblk, NT, 0, st>>>(qc, qp, sv.dim, R->sc, R->alpha, R->part, nullptr, R->coef, pprev);
        k_lz_beta<<<1, NT, 0, st>>>(R->sc, R->part, nblk, R->beta, R->dtype == HM_F64 ? LZ_TOL : LZ_TOL32);
    }
    HM_CUDA(cudaGetLastError());
    return HM_OK;
}

// raises the dynamic shared-memory limit of the product kernel (outside any capture)
template <class I, class T, class Acc>
static int prepare_t(const hm_basis *b) {
    HM_CUDA(raise_smem_limit(k_lz_matvec<I, T, Acc>, (int)row_smem_bytes<I>(b->view)));
    return HM_OK;
}

static int prepare(const hm_basis *b, int dtype) {
    const bool i64 = b->view.idx64 != 0;
    if (dtype == HM_F64) return i64 ? prepare_t<uint64_t, double, double>(b) : prepare_t<uint32_t, double, double>(b);
    return i64 ? prepare_t<uint64_t, float, float>(b) : prepare_t<uint32_t, float, float>(b);
}

static int enqueue_phase(hm_lanczos *R, int phase, cudaStream_t st) {
    const int parity = R->host_j & 1;
    const bool i64 = R->basis->view.idx64 != 0;
    int rc;
    if (R->dtype == HM_F64)
        rc = i64 ? enqueue_phase_t<uint64_t, double, double>(R, parity, phase, st)
                 : enqueue_phase_t<uint32_t, double, double>(R, parity, phase, st);
    else
        rc = i64 ? enqueue_phase_t<uint64_t, float, float>(R, parity, phase, st)
                 : enqueue_phase_t<uint32_t, float, float>(R, parity, phase, st);
    if (rc == HM_OK && phase == 1) R->host_j += 1;
    return rc;
}

static int enqueue_step(hm_lanczos *R, cudaStream_t st) {
    HM_TRY(enqueue_phase(R, 0, st));
    return enqueue_phase(R, 1, st);
}

// (re)starts the recurrence: q_cur = v0 (or seeded), q_prev = 0, sigma = 1/|v0|
static int enqueue_start(hm_lanczos *R, const void *v0, uint64_t seed, cudaStream_t st) {
    const SectorView &sv = R->basis->view;
    const size_t es = R->dtype == HM_F64 ? 8 : 4;
    void *b0 = R->work + R->L.buf[0];
    void *b1 = R->work + R->L.buf[1];
    if (v0) HM_CUDA(cudaMemcpyAsync(b0, v0, sv.dim * es, cudaMemcpyDeviceToDevice, st));
    else HM_TRY(start_vector_dev(sv.dim, seed, 0, b0, R->dtype, st));
    HM_CUDA(cudaMemsetAsync(b1, 0, sv.dim * es, st));
    HM_CUDA(cudaMemsetAsync(R->sc, 0, sizeof(LzScalars), st));
    if (R->use_blk) HM_CUDA(cudaMemsetAsync(R->hpart, 0, ((size_t)2 << R->blk.H) * sizeof(double), st));
    const int nblk = grid_blocks(sv.dim, NT);
    if (R->dtype == HM_F64) k_sumsq<double><<<nblk, NT, 0, st>>>((const double *)b0, sv.dim, R->part, &R->sc->emax[0]);
    else k_sumsq<float><<<nblk, NT, 0, st>>>((const float *)b0, sv.dim, R->part, nullptr);
    k_lz_start<<<1, NT, 0, st>>>(R->sc, R->part, nblk);
    if ((R->use_blk || R->use_s1) && R->dtype == HM_F64) {
        k_fix_start<<<nblk, NT, 0, st>>>((unsigned long long *)b0, (long long *)(R->work + R->L.xs[0]), sv.dim, R->sc,
                                         R->qqp);
    }
    HM_CUDA(cudaGetLastError());
    R->host_j = 0;
    R->next_phase = 0;
    return HM_OK;
}

static int lz_create(const hm_basis *b, int n_bonds, const int32_t *u, const int32_t *v,
                     const double *J, int dtype, int max_steps, void *work, size_t work_bytes,
                     bool grad, hm_lanczos **out) {
    if (!b || !out) return fail(HM_EINVAL, "NULL argument");
    if (dtype != HM_F64 && dtype != HM_F32) return fail(HM_EINVAL, "bad dtype");
    if (max_steps < 1 || max_steps > 100000) return fail(HM_EINVAL, "steps must be in 1..100000");
    hm_lanczos *R = new (std::nothrow) hm_lanczos();
    if (!R) return fail(HM_ENOMEM, "host allocation failed");
    int rc = make_bonds(b, n_bonds, u, v, J, &R->bp);
    if (rc < 0) { delete R; return rc; }
    R->basis = b;
    R->dtype = dtype;
    R->max_steps = max_steps;
    R->L = lz_layout(b, dtype, max_steps, grad, n_bonds);
    if (!work || work_bytes < R->L.total || ((uintptr_t)work & 255)) {
        size_t need = R->L.total;
        delete R;
        return fail(HM_EWORKSPACE, "workspace must be >= %zu bytes, 256-byte aligned", need);
    }
    rc = prepare(b, dtype);
    if (rc < 0) { delete R; return rc; }
    R->use_blk = 0;
    R->use_mom = b->mom_k >= 0;
    rc = R->use_mom ? 1 : blk_lz_plan(const_cast<hm_basis *>(b), R->bp, dtype, &R->blk, &R->blk_blocks);
    if (rc < 0) { delete R; return rc; }
    // the per-block partials were sized for 2^hpart_H blocks
    R->use_blk = rc == 0 && (dtype == HM_F32 || R->L.shadow) && R->L.hpart != 0 && R->blk.H <= R->L.hpart_H &&
                 R->blk.H <= 17;
    R->jit = nullptr;
    R->run = row_run_len();
    if (R->use_blk) {
        int jb = 0;
        const void *jk = nullptr;
        rc = blk_target_table(const_cast<hm_basis *>(b), &R->blk, dtype == HM_F64 ? 8 : 4);
        if (rc < 0) { delete R; return rc; }
        if (blk_lz_jit(R->blk, dtype, R->bp, &jk, &jb) == 0) { R->jit = jk; R->blk_blocks = jb; }
        if (R->blk.perbond && !R->jit) R->use_blk = 0;   // per-bond rows run only specialised
    }
    R->split = 0;
    R->jit2 = nullptr;
    if (R->use_blk && R->jit && R->L.shadow) {
        BlkParams pa, pb;
        const void *ka = nullptr, *kb = nullptr;
        int na = 0, nb2 = 0;
        if (blk_lz_split(const_cast<hm_basis *>(b), R->bp, R->blk, dtype, &pa, &pb, &ka, &kb, &na, &nb2) == 0) {
            R->blk = pa; R->jit = ka; R->blk_blocks = na;
            R->blk2 = pb; R->jit2 = kb; R->blk_blocks2 = nb2;
            R->split = 1;
        }
    }
    R->use_s1 = 0;
    if (!R->use_blk && !R->use_mom && R->L.s1part) {
        rc = s1_plan(const_cast<hm_basis *>(b), R->bp, &R->s1);
        if (rc < 0) { delete R; return rc; }
        R->use_s1 = rc == 0 && (uint64_t)R->s1.nblocks <= R->L.s1n;
        // FP64 runs only specialised (and with the fixed-point copies); FP32 compiles its
        // specialised kernel here, outside any graph capture (the generic one serves without)
        if (R->use_s1 && dtype == HM_F64) R->use_s1 = R->L.shadow && s1_jit_ready(R->s1, 2);
        else if (R->use_s1) (void)s1_jit_ready(R->s1, 1);
    }
    if (b->parity && !R->use_blk) {
        delete R;
        return fail(HM_EINVAL, "spin-flip basis: this bond list does not take the s = 1/2 block path");
    }
    R->work = (unsigned char *)work;
    R->sc = (LzScalars *)(R->work + R->L.sc);
    R->alpha = (double *)(R->work + R->L.alpha);
    R->beta = (double *)(R->work + R->L.beta);
    R->part = (double *)(R->work + R->L.part);
    R->hpart = R->L.hpart ? (double *)(R->work + R->L.hpart) : nullptr;
    R->qqp = R->L.shadow ? (double *)(R->work + R->L.qqp) : nullptr;
    R->psi = nullptr;
    R->coef = grad ? (double *)(R->work + R->L.coef) : nullptr;
    *out = R;
    return HM_OK;
}

// steps launched as one captured graph (the recurrence state lives on the device, so
// no host round trip is needed between steps)
static int run_steps_graph(hm_lanczos *R, int steps, cudaStream_t st) {
    cudaStream_t cap;
    HM_CUDA(cudaStreamCreateWithFlags(&cap, cudaStreamNonBlocking));
    cudaGraph_t g = nullptr;
    cudaGraphExec_t ge = nullptr;
    int rc = HM_OK;
    cudaError_t e = cudaStreamBeginCapture(cap, cudaStreamCaptureModeThreadLocal);
    if (e == cudaSuccess) {
        for (int k = 0; k < steps && rc == HM_OK; ++k) rc = enqueue_step(R, cap);
        cudaError_t e2 = cudaStreamEndCapture(cap, &g);
        if (rc == HM_OK && e2 != cudaSuccess) rc = cuda_fail(e2, "cudaStreamEndCapture");
    } else {
        rc = cuda_fail(e, "cudaStreamBeginCapture");
    }
    if (rc == HM_OK) {
        e = cudaGraphInstantiate(&ge, g, 0);
        if (e != cudaSuccess) rc = cuda_fail(e, "cudaGraphInstantiate");
    }
    if (rc == HM_OK) {
        e = cudaGraphLaunch(ge, st);
        if (e != cudaSuccess) rc = cuda_fail(e, "cudaGraphLaunch");
    }
    if (ge) cudaGraphExecDestroy(ge);
    if (g) cudaGraphDestroy(g);
    cudaStreamDestroy(cap);
    return rc;
}

// lowest Ritz value, steps done and status of one run (device, out[0..2]); NaN without steps
__global__ void k_branch_out(const LzScalars *S, const double *alpha, const double *beta, double *out) {
    if (threadIdx.x != 0 || blockIdx.x != 0) return;
    const int m = S->j;
    out[0] = m >= 1 ? tri_eig(m, alpha, beta, 1) : __longlong_as_double(0x7ff8000000000000ll);
    out[1] = (double)m;
    out[2] = (double)S->status;
}

size_t lz_run_workspace(const hm_basis *b, int dtype, int steps) { return lz_layout(b, dtype, steps, false, 0).total; }

// One Lanczos run per basis, each from the uniform start vector of its seed, each on a branch
// of its own in one captured graph that is launched once on st (the branches are
// independent, so small runs overlap on the GPU).  Run i uses work[offs[i], offs[i] + its
// workspace) and leaves its lowest Ritz value, steps done and status in out[3i .. 3i+2]
// (device).  Everything is planned (and specialised kernels compiled) before the capture;
// st is synchronised once, after the graph, before this returns.
int lz_branches(const std::vector<const hm_basis *> &bases, int n_bonds, const int32_t *u, const int32_t *v,
                const double *J, const std::vector<uint64_t> &seeds, int steps, int dtype, unsigned char *work,
                const std::vector<size_t> &offs, double *out, cudaStream_t st) {
    const int n = (int)bases.size();
    std::vector<hm_lanczos *> runs(n, nullptr);
    std::vector<cudaStream_t> br(n, nullptr);
    std::vector<cudaEvent_t> done(n, nullptr);
    cudaEvent_t fork = nullptr;
    cudaStream_t cap = nullptr;
    cudaGraph_t g = nullptr;
    cudaGraphExec_t ge = nullptr;
    int rc = HM_OK;
    for (int i = 0; i < n && rc == HM_OK; ++i)
        rc = lz_create(bases[i], n_bonds, u, v, J, dtype, steps, work + offs[i], lz_run_workspace(bases[i], dtype, steps),
                       false, &runs[i]);
    cudaError_t e = cudaSuccess;
    if (rc == HM_OK && (e = cudaStreamCreateWithFlags(&cap, cudaStreamNonBlocking)) != cudaSuccess) rc = cuda_fail(e, "stream");
    if (rc == HM_OK && (e = cudaEventCreateWithFlags(&fork, cudaEventDisableTiming)) != cudaSuccess) rc = cuda_fail(e, "event");
    for (int i = 0; i < n && rc == HM_OK; ++i) {
        if ((e = cudaStreamCreateWithFlags(&br[i], cudaStreamNonBlocking)) != cudaSuccess) rc = cuda_fail(e, "stream");
        else if ((e = cudaEventCreateWithFlags(&done[i], cudaEventDisableTiming)) != cudaSuccess) rc = cuda_fail(e, "event");
    }
    if (rc == HM_OK) {
        e = cudaStreamBeginCapture(cap, cudaStreamCaptureModeThreadLocal);
        if (e != cudaSuccess) rc = cuda_fail(e, "cudaStreamBeginCapture");
        else {
            if ((e = cudaEventRecord(fork, cap)) != cudaSuccess) rc = cuda_fail(e, "fork");
            for (int i = 0; i < n && rc == HM_OK; ++i) {
                if ((e = cudaStreamWaitEvent(br[i], fork, 0)) != cudaSuccess) { rc = cuda_fail(e, "branch"); break; }
                rc = enqueue_start(runs[i], nullptr, seeds[i], br[i]);
                for (int k = 0; k < steps && rc == HM_OK; ++k) rc = enqueue_step(runs[i], br[i]);
                if (rc != HM_OK) break;
                k_branch_out<<<1, 32, 0, br[i]>>>(runs[i]->sc, runs[i]->alpha, runs[i]->beta, out + 3 * i);
                if ((e = cudaGetLastError()) != cudaSuccess) { rc = cuda_fail(e, "k_branch_out"); break; }
                if ((e = cudaEventRecord(done[i], br[i])) != cudaSuccess || (e = cudaStreamWaitEvent(cap, done[i], 0)) != cudaSuccess)
                    rc = cuda_fail(e, "join");
            }
            cudaError_t e2 = cudaStreamEndCapture(cap, &g);
            if (rc == HM_OK && e2 != cudaSuccess) rc = cuda_fail(e2, "cudaStreamEndCapture");
        }
    }
    if (rc == HM_OK && (e = cudaGraphInstantiate(&ge, g, 0)) != cudaSuccess) rc = cuda_fail(e, "cudaGraphInstantiate");
    if (rc == HM_OK && (e = cudaGraphLaunch(ge, st)) != cudaSuccess) rc = cuda_fail(e, "cudaGraphLaunch");
    if (rc == HM_OK && (e = cudaStreamSynchronize(st)) != cudaSuccess) rc = cuda_fail(e, "sectors");
    if (ge) cudaGraphExecDestroy(ge);
    if (g) cudaGraphDestroy(g);
    for (int i = 0; i < n; ++i) {
        if (done[i]) cudaEventDestroy(done[i]);
        if (br[i]) cudaStreamDestroy(br[i]);
        delete runs[i];
    }
    if (fork) cudaEventDestroy(fork);
    if (cap) cudaStreamDestroy(cap);
    return rc;
}

}  // namespace hm

using namespace hm;

extern "C" {

int lanczos_workspace(const hm_basis *b, int dtype, int max_steps, size_t *bytes) {
    if (!b || !bytes) return fail(HM_EINVAL, "NULL argument");
    if (dtype != HM_F64 && dtype != HM_F32) return fail(HM_EINVAL, "bad dtype");
    if (max_steps < 1) return fail(HM_EINVAL, "max_steps must be >= 1");
    *bytes = lz_layout(b, dtype, max_steps, false, 0).total;
    return HM_OK;
}

int e0_grad_workspace(const hm_basis *b, int n_bonds, int steps, size_t *bytes) {
    if (!b || !bytes) return fail(HM_EINVAL, "NULL argument");
    if (steps < 1) return fail(HM_EINVAL, "steps must be >= 1");
    *bytes = lz_layout(b, HM_F64, steps, true, n_bonds).total;
    return HM_OK;
}

int lanczos_init(const hm_basis *b, int n_bonds, const int32_t *u, const int32_t *v,
                 const double *J, const void *v0, uint64_t seed, int dtype, int max_steps,
                 void *work, size_t work_bytes, void *stream, hm_lanczos **out) {
    if (out) *out = nullptr;
    hm_lanczos *R = nullptr;
    HM_TRY(lz_create(b, n_bonds, u, v, J, dtype, max_steps, work, work_bytes, false, &R));
    int rc = enqueue_start(R, v0, seed, as_stream(stream));
    if (rc < 0) { delete R; return rc; }
    *out = R;
    return HM_OK;
}

int lanczos_step(hm_lanczos *R, void *stream) {
    if (!R) return fail(HM_EINVAL, "run is NULL");
    if (R->host_j >= R->max_steps) return fail(HM_EINVAL, "max_steps (%d) reached", R->max_steps);
    if (R->next_phase != 0) return fail(HM_EINVAL, "a step is half done (phase 1 pending)");
    return enqueue_step(R, as_stream(stream));
}

int lanczos_substep(hm_lanczos *R, int phase, void *stream) {
    if (!R) return fail(HM_EINVAL, "run is NULL");
    if (phase != 0 && phase != 1) return fail(HM_EINVAL, "phase must be 0 or 1");
    if (phase != R->next_phase) return fail(HM_EINVAL, "phases must alternate 0, 1, 0, ...");
    if (R->host_j >= R->max_steps) return fail(HM_EINVAL, "max_steps (%d) reached", R->max_steps);
    HM_TRY(enqueue_phase(R, phase, as_stream(stream)));
    R->next_phase = 1 - phase;
    return HM_OK;
}

int lanczos_read(hm_lanczos *R, double *alpha, double *beta, int *steps_done, void *stream) {
    if (!R) return fail(HM_EINVAL, "run is NULL");
    cudaStream_t st = as_stream(stream);
    LzScalars S;
    HM_CUDA(cudaMemcpyAsync(&S, R->sc, sizeof S, cudaMemcpyDeviceToHost, st));
    HM_CUDA(cudaStreamSynchronize(st));
    if (steps_done) *steps_done = S.j;
    if (alpha && S.j > 0) HM_CUDA(cudaMemcpy(alpha, R->alpha, S.j * 8, cudaMemcpyDeviceToHost));
    if (beta && S.j > 0) HM_CUDA(cudaMemcpy(beta, R->beta, S.j * 8, cudaMemcpyDeviceToHost));
    if (S.status < 0) return fail(S.status, "Lanczos start vector has zero norm");
    return S.status;
}

int lanczos_free(hm_lanczos *R) {
    delete R;
    return HM_OK;
}

int lanczos_kernel_name(const hm_lanczos *R, char *name, int cap) {
    if (!R || !name || cap < 1) return fail(HM_EINVAL, "NULL argument");
    const bool f64 = R->dtype == HM_F64;
    const char *n = R->use_mom ? "k_mom_matvec"
                    : R->use_s1 ? s1_kernel_name(R->s1, f64 ? 2 : 1)
                    : !R->use_blk ? "k_lz_matvec"
                    : R->split  ? "k_blk_lz64a_jit+k_blk_lz64b_jit"
                    : R->jit    ? (f64 ? "k_blk_lz64_jit" : "k_blk_lz32_jit")
                                : (f64 ? "k_blk_lz64" : "k_blk_lz32");
    snprintf(name, (size_t)cap, "%s", n);
    return HM_OK;
}

int lanczos_run(const hm_basis *b, int n_bonds, const int32_t *u, const int32_t *v,
                const double *J, const void *v0, uint64_t seed, int steps, int dtype,
                void *work, size_t work_bytes, double *alpha, double *beta, int *steps_done,
                double *ritz, int n_ritz, void *stream) {
    if (n_ritz < 0 || n_ritz > 64 || (n_ritz > 0 && !ritz)) return fail(HM_EINVAL, "n_ritz must be in 0..64");
    hm_lanczos *R = nullptr;
    HM_TRY(lanczos_init(b, n_bonds, u, v, J, v0, seed, dtype, steps, work, work_bytes, stream, &R));
    cudaStream_t st = as_stream(stream);
    int rc = run_steps_graph(R, steps, st);
    double *d_ritz = (double *)(R->work + R->L.ritz);
    if (rc == HM_OK && n_ritz > 0) {
        k_ritz<<<1, 64, 0, st>>>(R->sc, R->alpha, R->beta, n_ritz, d_ritz);
        cudaError_t e = cudaGetLastError();
        if (e != cudaSuccess) rc = cuda_fail(e, "k_ritz");
    }
    if (rc == HM_OK) rc = lanczos_read(R, alpha, beta, steps_done, stream);
    if (rc >= 0 && n_ritz > 0) {
        cudaError_t e = cudaMemcpy(ritz, d_ritz, n_ritz * 8, cudaMemcpyDeviceToHost);
        if (e != cudaSuccess) rc = cuda_fail(e, "ritz copy");
    }
    delete R;
    return rc;
}

int e0_grad(const hm_basis *b, int n_bonds, const int32_t *u, const int32_t *v, const double *J,
            const void *v0, uint64_t seed, int steps, void *work, size_t work_bytes, double *e0,
            double *dE0_dJ, double *psi_out, void *stream) {
    if (b && b->parity) return fail(HM_EINVAL, "e0_grad: not available on a spin-flip basis");
    if (b && b->mom_k >= 0) return fail(HM_EINVAL, "e0_grad: not available on a momentum basis");
    if (!e0 || (n_bonds > 0 && !dE0_dJ)) return fail(HM_EINVAL, "NULL output");
    hm_lanczos *R = nullptr;
    HM_TRY(lz_create(b, n_bonds, u, v, J, HM_F64, steps, work, work_bytes, true, &R));
    cudaStream_t st = as_stream(stream);
    const SectorView &sv = b->view;
    const int nblk = grid_blocks(sv.dim, NT);
    double *d_ritz = (double *)(R->work + R->L.ritz);
    double *tri = (double *)(R->work + R->L.tri);
    double *res = (double *)(R->work + R->L.res);
    int rc = HM_OK;
    // pass 1: T
    rc = enqueue_start(R, v0, seed, st);
    for (int k = 0; k < steps && rc == HM_OK; ++k) rc = enqueue_step(R, st);
    if (rc == HM_OK) {
        // residual of the lowest Ritz pair of every leading T_k, then the shortest
        // converged length and the eigenvector of T there (no ghost copies yet)
        k_conv_scan<<<(steps + 63) / 64, 64, 0, st>>>(R->sc, R->alpha, R->beta, tri, steps, res);
        k_pick_and_vec<<<1, 1, 0, st>>>(R->sc, R->alpha, R->beta, tri, steps, res, 1e-10, R->coef, d_ritz);
        cudaError_t e = cudaGetLastError();
        if (e != cudaSuccess) rc = cuda_fail(e, "e0_grad: eigenvector");
    }
    // pass 2: the same recurrence from the same start, accumulating psi = sum_j c_j v_j
    LzScalars S1{};
    if (rc == HM_OK) {
        cudaError_t e = cudaMemcpyAsync(&S1, R->sc, sizeof S1, cudaMemcpyDeviceToHost, st);
        if (e == cudaSuccess) e = cudaStreamSynchronize(st);
        if (e != cudaSuccess) rc = cuda_fail(e, "e0_grad: read pass 1");
        if (rc == HM_OK && S1.status < 0) rc = fail(S1.status, "Lanczos start vector has zero norm");
    }
    if (rc == HM_OK) {
        R->psi = (double *)(R->work + R->L.psi);
        cudaError_t e = cudaMemsetAsync(R->psi, 0, sv.dim * 8, st);
        if (e != cudaSuccess) rc = cuda_fail(e, "memset psi");
        if (rc == HM_OK) rc = enqueue_start(R, v0, seed, st);
        for (int k = 0; k < S1.mconv && rc == HM_OK; ++k) rc = enqueue_step(R, st);
    }
    if (rc == HM_OK) {
        k_sumsq<double><<<nblk, NT, 0, st>>>(R->psi, sv.dim, R->part, nullptr);
        k_store_nrm2<<<1, NT, 0, st>>>(R->sc, R->part, nblk);
        cudaError_t e = cudaGetLastError();
        if (e != cudaSuccess) rc = cuda_fail(e, "e0_grad: norm");
    }
    // dE0/dJ_b = -<psi| s_u.s_v |psi> / <psi|psi>
    double *d_out = (double *)(R->work + R->L.gout);
    if (rc == HM_OK && n_bonds > 0) {
        std::vector<double> ones(n_bonds, 1.0);
        BondParams bp1;
        rc = make_bonds(b, n_bonds, u, v, ones.data(), &bp1);
        if (rc == HM_OK)
            rc = bond_corr_dev(b, bp1, R->psi, R->psi, d_out, HM_F64, R->work + R->L.bpart,
                               bond_corr_bytes(b, n_bonds), -1.0, &R->sc->nrm2, st);
    }
    if (rc == HM_OK && psi_out) {
        k_scale<<<nblk, NT, 0, st>>>(R->psi, sv.dim, R->sc);
        cudaError_t e = cudaMemcpyAsync(psi_out, R->psi, sv.dim * 8, cudaMemcpyDeviceToDevice, st);
        if (e != cudaSuccess) rc = cuda_fail(e, "psi copy");
    }
    double rz[2] = {0, 0};
    if (rc == HM_OK) {
        cudaError_t e = cudaMemcpyAsync(rz, d_ritz, 16, cudaMemcpyDeviceToHost, st);
        if (e == cudaSuccess && n_bonds > 0) e = cudaMemcpyAsync(dE0_dJ, d_out, n_bonds * 8, cudaMemcpyDeviceToHost, st);
        if (e == cudaSuccess) e = cudaStreamSynchronize(st);
        if (e != cudaSuccess) rc = cuda_fail(e, "e0_grad: results");
    }
    delete R;
    if (rc < 0) return rc;
    *e0 = rz[0];
    if (std::isfinite(rz[1]) && rz[1] - rz[0] < 1e-8 * std::fabs(rz[0])) return HM_DEGENERATE;
    return HM_OK;
}

}  // extern "C"
