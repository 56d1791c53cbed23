// ftlm.cu -- finite-temperature Lanczos over all sectors of an s = 1/2 system in one
// persistent, cooperative launch (Jaklic and Prelovsek's estimator; the paper cites it
// as an application of the Lanczos machinery, Sec. 1).
//
// For every sector A (digit sum, M = N/2 - A) and start vector r = 0..R-1 a Lanczos run
// of up to `steps` steps starts from the +-1 vector of SplitMix64 stream (seed, A, r).
// All R runs of a sector share one product: a row's R vector entries sit in one
// 128-byte line (row-major [dim][32]), a warp serves VT rows with 32/VT lanes each, lane
// l of a row holding vectors l*VT .. l*VT+VT-1, so the codec of a row runs once per
// warp instruction for all of its vectors.  The rows of all sectors are cut into the
// blocks of blk.cuh (one high word, all low words).  Every warp owns an equal share of
// the rows (a fixed interval of the row order, cut on the host): it walks the blocks its
// rows fall in, builds their exchange lists itself and writes one partial sum per sector
// it touches, so no CTA barrier separates blocks and the sums come out in a fixed order.
// A step is four phases separated by grid barriers with bounded waits:
//   A  u = sigma H q - beta_prev sigma_prev q_prev over q_prev, alpha partials
//   B  alpha per (sector, vector): the sector's warp partials in order
//   C  w = u - alpha sigma q over q_prev, |w|^2 partials
//   D  beta, breakdown, sigma
// Then per (sector, vector) the tridiagonal T is diagonalised on the device (implicit
// symmetric QR with Wilkinson shifts, Golub and Van Loan, Matrix Computations, Sec. 8.3),
// keeping the first row of the eigenvector matrix: Ritz values theta_j and weights
// tau_j = (first component)^2.  Finally
//   Z(T) = sum_A (D_A / R) sum_r sum_j tau e^{-(theta - e_ref)/T},
//   E(T) = [same with theta inside] / Z(T)     (Z returned relative to e^{-e_ref/T}).
#include <algorithm>
#include <cstdlib>
#include <climits>
#include <cmath>
#include <cstring>
#include <map>
#include <vector>

#include "blk.cuh"

namespace hm {

__host__ __device__ __forceinline__ size_t al16f(size_t x) { return (x + 15) & ~(size_t)15; }

constexpr int FT_NT = 512;          // threads per CTA of the persistent kernel
// CTAs per SM the register budget is cut for: three (40 registers; the widest tiling then
// spills a little) ran the N = 24 run in 825 ms against 989 ms with two (64 registers): the
// kernel waits on gather latency, and the extra resident warps hide more of it
#ifndef HM_FT_CTAS
#define HM_FT_CTAS 3
#endif
constexpr int FT_CTAS = HM_FT_CTAS;
constexpr int FT_W = 32;            // row stride in floats (vectors per row, padded)
constexpr int FT_MAXS = 65;         // sectors (N + 1 for s = 1/2, N <= 64)
constexpr double FT_TOL = 1e-5;     // breakdown threshold (above the FP32 noise floor)

struct GridBar {
    unsigned count;
    unsigned gen;
    int abort;
    int pad;
};

// A warp's share of the row phases: global rows [g0, g1) (all sectors' rows in order, which
// is also the order of the blocks in `items`), the first of them in item it0; its partial
// sums go to slots slot0, slot0 + 1, ... one per sector the rows touch, so the slots of a
// sector are consecutive over the warps.
struct FtRange {
    uint64_t g0, g1;
    uint32_t it0, slot0;
};

struct FtDev {
    // per (sector, vector) state, index s * FT_W + v
    double *sig_cur, *sig_prev, *beta_prev, *scale, *as;
    int *done, *nsteps;
    double *alpha, *beta;           // [(s * FT_W + v) * steps + j]
    double *part;                   // [slot][v]: warp partials of the update phase (FtRange)
    double *parta;                  // [sector][warp][v]: warp partials of the product phase
    double *partc;                  // [sector][cta][v]: the same summed over each CTA's warps
    const uint32_t *ck_it0;         // [chunk]: the block holding the chunk's first row
    const uint32_t *ck_cs;          // [nsec + 1]: sector s owns chunks ck_cs[s] .. ck_cs[s + 1] - 1
    const FtRange *wr;              // [warp]
    const uint32_t *slo;            // [nsec + 1]: sector s owns slots slo[s] .. slo[s + 1] - 1
    int *sec_active;                // [s]
    GridBar *bar;
    const uint32_t *items;          // (A << 16) | h, sorted by A
    const uint64_t *rowoff;         // first global row of sector A
    const uint32_t *secdim;         // D(N, A)
    float *q0, *q1;                 // [rows][FT_W]
    double *theta, *tau;            // [(s * FT_W + v) * steps + j]
    int *mlen;                      // Krylov length per (s, v)
    double *zsum, *esum, *eref;     // thermodynamics (n_t each), e_ref
};

// A sector whose dimension does not exceed the step count would exhaust its Krylov
// space; it is diagonalised exactly instead (dense, FP64, one CTA): the Lanczos
// quadrature sum_j tau_j f(theta_j) of a start vector is then the exact <r|f(H)|r>.
struct ExactSec {
    int A, dim;
    uint32_t cd_off;                // its CD table inside the exact-table buffer
    int cd_rowlen, cd_len;
    uint64_t mat_off;               // doubles: H (dim x dim) then V (dim x dim)
};
constexpr int FT_MAXEXACT = 40;

struct FtParams {
    BlkParams P;                    // block plan built with A = N (full binomial table)
    FtDev d;
    int nsec, R, steps, nitems;
    uint32_t nchunks, ck_rows;      // product phase: chunks of ck_rows rows (a sector's last is shorter)
    unsigned nctas;
    uint64_t seed;
    unsigned long long barrier_ns;  // a grid barrier gives up after this long (default 5 s)
    uint64_t exact_mask;            // bit A set: sector A is diagonalised exactly
    int nexact;
    ExactSec ex[FT_MAXEXACT];
};

__device__ __forceinline__ unsigned long long globaltimer_ns() {
    unsigned long long t;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
    return t;
}

// grid-wide barrier of a cooperative launch; gives up after limit_ns (sets abort) so a
// lost CTA can never hang the GPU
__device__ bool grid_sync(GridBar *gb, unsigned nctas, unsigned long long limit_ns) {
    __syncthreads();
    if (threadIdx.x == 0) {
        volatile unsigned *vgen = &gb->gen;
        volatile int *vab = &gb->abort;
        const unsigned g = *vgen;
        __threadfence();
        const unsigned arrived = atomicAdd(&gb->count, 1u);
        if (arrived == nctas - 1) {
            atomicExch(&gb->count, 0u);
            __threadfence();
            atomicAdd(&gb->gen, 1u);
        } else {
            const unsigned long long t0 = globaltimer_ns();
            while (*vgen == g) {
                if (*vab) break;
                if (globaltimer_ns() - t0 > limit_ns) { atomicExch(&gb->abort, 1); break; }
                __nanosleep(200);
            }
        }
        __threadfence();
    }
    __syncthreads();
    return *(volatile int *)&gb->abort == 0;
}

// ---- start vectors and state -----------------------------------------------------------
__global__ void k_ft_init(FtParams F) {
    const FtDev &d = F.d;
    const uint64_t nrows = d.rowoff[F.nsec];
    const uint64_t total = nrows * FT_W;
    for (uint64_t t = blockIdx.x * (uint64_t)blockDim.x + threadIdx.x; t < total;
         t += (uint64_t)gridDim.x * blockDim.x) {
        const uint64_t row = t / FT_W;
        const int v = (int)(t % FT_W);
        int A = 0;
        while (d.rowoff[A + 1] <= row) ++A;          // few sectors: linear search
        float val = 0.0f;
        if (v < F.R) {
            const uint64_t stream = sm64(F.seed, ((uint64_t)A << 20) + (uint64_t)v);
            val = (sm64(stream, row - d.rowoff[A]) >> 63) ? -1.0f : 1.0f;
        }
        d.q0[t] = val;
        d.q1[t] = 0.0f;
    }
    // product-phase partials: the (sector, warp) pairs no chunk visits stay zero
    const uint64_t npa = (uint64_t)F.nsec * F.nctas * (FT_NT / 32) * FT_W;
    for (uint64_t t = blockIdx.x * (uint64_t)blockDim.x + threadIdx.x; t < npa; t += (uint64_t)gridDim.x * blockDim.x)
        d.parta[t] = 0.0;
    const int nst = F.nsec * FT_W;
    for (int t = blockIdx.x * blockDim.x + threadIdx.x; t < nst; t += gridDim.x * blockDim.x) {
        const int s = t / FT_W, v = t % FT_W;
        const bool on = v < F.R && d.secdim[s] > 0 && !((F.exact_mask >> s) & 1ull);
        d.sig_cur[t] = on ? 1.0 / sqrt((double)d.secdim[s]) : 0.0;   // |+-1 vector| = sqrt(dim)
        d.sig_prev[t] = 0.0;
        d.beta_prev[t] = 0.0;
        d.scale[t] = 0.0;
        d.as[t] = 0.0;
        d.done[t] = on ? 0 : 1;
        d.nsteps[t] = 0;
        d.mlen[t] = 0;
    }
    if (blockIdx.x == 0 && threadIdx.x < FT_MAXS && (int)threadIdx.x < F.nsec)
        d.sec_active[threadIdx.x] = ((F.exact_mask >> threadIdx.x) & 1ull) ? 0 : 1;
    if (blockIdx.x == 0 && threadIdx.x == 0) { d.bar->count = 0; d.bar->gen = 0; d.bar->abort = 0; }
}

// The warp's partials p[q] (vectors v0 + q of row group grp) summed over its VT row groups
// in a fixed order and written to slot `slot` of part, then cleared.  All 32 lanes call it.
template <int VT>
__device__ __forceinline__ void ft_warp_flush(ef::df *p, double *part, uint32_t slot, int lane, int grp, int v0) {
    constexpr int LPR = 32 / VT;                  // lanes per row group
#pragma unroll
    for (int q = 0; q < VT; ++q) {
        ef::df s = p[q];
#pragma unroll
        for (int g = 1; g < VT; ++g) {
            const float hi = __shfl_sync(0xffffffffu, p[q].hi, lane + g * LPR);
            const float lo = __shfl_sync(0xffffffffu, p[q].lo, lane + g * LPR);
            s = ef::df_add(s, ef::df{hi, lo});
        }
        if (grp == 0) part[(size_t)slot * FT_W + v0 + q] = (double)s.hi + (double)s.lo;
        p[q] = ef::df{0.0f, 0.0f};
    }
}

// Hop lists of block (h, k) for one warp: the valid high exchanges as row offsets,
// compacted by class (lane e tests bonds e and e + 32, ballots give the positions), and
// the targets of the cross exchanges.  The caller syncs the warp before and after.
__device__ __forceinline__ void ft_warp_setup(const BlkParams &P, const BlkTabs &tb, uint32_t h, int k, uint32_t off,
                                              const BlkShared &sh, int lane) {
    int val[2] = {0, 0}, hoff[2] = {0, 0};
#pragma unroll
    for (int half = 0; half < 2; ++half) {
        const int e = lane + 32 * half;
        if (e < P.nhb) {
            const int p = P.hb_p[e], q = P.hb_q[e];
            val[half] = (((h >> p) ^ (h >> q)) & 1u) ? 1 : 0;
            if (val[half]) hoff[half] = (int)(blk_off(P, tb, h ^ ((1u << p) | (1u << q)), k) - off);
        }
    }
    const uint32_t b0 = __ballot_sync(0xffffffffu, val[0]), b1 = __ballot_sync(0xffffffffu, val[1]);
    const uint32_t below = (1u << lane) - 1u;
    if (val[0]) sh.hcd[__popc(b0 & below)] = hoff[0];
    if (val[1]) sh.hcd[__popc(b0) + __popc(b1 & below)] = hoff[1];
    if (lane <= HM_BLK_MAXC) {                    // class c starts at the valid ones before hb_start[c]
        const int e = P.hb_start[lane];
        sh.hcs[lane] = e >= 32 ? __popc(b0) + __popc(e >= 64 ? b1 : b1 & ((1u << (e - 32)) - 1u))
                               : __popc(b0 & ((1u << e) - 1u));
    }
    for (int e = lane; e < P.ncb; e += 32) {
        const int q = P.cb_q[e];
        const uint32_t bq = (h >> q) & 1u;
        const int k2 = k + (bq ? 1 : -1);
        const bool ok = k2 >= 0 && k2 <= P.K;
        sh.cbq[e] = (uint8_t)bq;
        sh.ck[e] = (int8_t)(ok ? k2 : -1);
        sh.coff[e] = ok ? blk_off(P, tb, h ^ (1u << q), k2) : 0u;
    }
}

// Per (sector, vector) sums of the warp partials: the slots of sector s, slo[s] ..
// slo[s + 1] - 1, in a fixed order (16 strided chunks, then the chunks in order);
// f(s, v, sum) runs on warp 0 of the CTA that owns sector s.  All threads call it.
template <class F>
__device__ __forceinline__ void ft_sector_sums(const FtParams &Fp, double *red, F &&f) {
    const FtDev &d = Fp.d;
    constexpr int NCH = FT_NT / FT_W;
    const int v = threadIdx.x % FT_W, c = threadIdx.x / FT_W;
    for (int s = blockIdx.x; s < Fp.nsec; s += gridDim.x) {
        const uint32_t s0 = d.slo[s], s1 = d.slo[s + 1];
        double a0 = 0.0, a1 = 0.0, a2 = 0.0, a3 = 0.0;
        uint32_t sl = s0 + c;
        for (; sl + 3 * NCH < s1; sl += 4 * NCH) {
            a0 += d.part[(size_t)sl * FT_W + v];
            a1 += d.part[(size_t)(sl + NCH) * FT_W + v];
            a2 += d.part[(size_t)(sl + 2 * NCH) * FT_W + v];
            a3 += d.part[(size_t)(sl + 3 * NCH) * FT_W + v];
        }
        for (; sl < s1; sl += NCH) a0 += d.part[(size_t)sl * FT_W + v];
        const double a = (a0 + a1) + (a2 + a3);
        red[c * FT_W + v] = a;
        __syncthreads();
        if (c == 0) {
            double t = 0.0;
            for (int i = 0; i < NCH; ++i) t += red[i * FT_W + v];
            f(s, v, t);
        }
        __syncthreads();
    }
}

// Per (sector, vector) sums of the product-phase partials partc[s][b][v] over all CTAs b
// in a fixed order (16 strided chunks of four running sums, then the chunks in order);
// f(s, v, sum) runs on warp 0 of the CTA that owns sector s.  All threads call it.
template <class F>
__device__ __forceinline__ void ft_sector_sums_a(const FtParams &Fp, double *red, F &&f) {
    const FtDev &d = Fp.d;
    constexpr int NCH = FT_NT / FT_W;
    const int v = threadIdx.x % FT_W, c = threadIdx.x / FT_W;
    const unsigned nb = Fp.nctas;
    for (int s = blockIdx.x; s < Fp.nsec; s += gridDim.x) {
        const double *ps = d.partc + (size_t)s * nb * FT_W;
        double a0 = 0.0, a1 = 0.0, a2 = 0.0, a3 = 0.0;
        unsigned b = c;
        for (; b + 3 * NCH < nb; b += 4 * NCH) {
            a0 += ps[(size_t)b * FT_W + v];
            a1 += ps[(size_t)(b + NCH) * FT_W + v];
            a2 += ps[(size_t)(b + 2 * NCH) * FT_W + v];
            a3 += ps[(size_t)(b + 3 * NCH) * FT_W + v];
        }
        for (; b < nb; b += NCH) a0 += ps[(size_t)b * FT_W + v];
        const double a = (a0 + a1) + (a2 + a3);
        red[c * FT_W + v] = a;
        __syncthreads();
        if (c == 0) {
            double t = 0.0;
            for (int i = 0; i < NCH; ++i) t += red[i * FT_W + v];
            f(s, v, t);
        }
        __syncthreads();
    }
}

// VT consecutive floats of one row (16- or 8-byte aligned for VT = 4, 2), read-only path
template <int VT>
__device__ __forceinline__ void ft_ld(const float *p, float *v) {
    if constexpr (VT == 4) {
        const float4 t = __ldg((const float4 *)p);
        v[0] = t.x; v[1] = t.y; v[2] = t.z; v[3] = t.w;
    } else if constexpr (VT == 2) {
        const float2 t = __ldg((const float2 *)p);
        v[0] = t.x; v[1] = t.y;
    } else {
        v[0] = __ldg(p);
    }
}

// sector of a global row (few sectors: linear search)
__device__ __forceinline__ int ft_sector_of(const FtDev &d, int nsec, uint64_t g) {
    int A = 0;
    while (A + 1 < nsec && d.rowoff[A + 1] <= g) ++A;
    return A;
}

// per-warp shared slice: hop lists | sigma, gamma of the current sector | alpha sigma
__host__ __device__ __forceinline__ size_t ft_warp_bytes(int max_block) {
    return al16f(blk_shared_bytes(max_block)) + al16f(FT_W * 4 * 3);
}

// ---- the persistent kernel ---------------------------------------------------------------
// Every warp owns the global rows [g0, g1) of its FtRange (rows of all sectors in order,
// balanced over the warps) in both row phases, so no CTA barrier separates blocks: a
// warp walks the blocks its rows fall in, builds their hop lists itself, and writes one
// partial per sector it touches.  Shared layout: block tables | per-warp slices | the
// sector-sum scratch.  A block's own rows are read through L1.
template <int NC, int VT>
__global__ void __launch_bounds__(FT_NT, FT_CTAS) k_ftlm(FtParams F) {
    const BlkParams &P = F.P;
    const FtDev &d = F.d;
    extern __shared__ __align__(16) unsigned char smem[];
    const BlkTabs tb = stage_blk_tables(P, smem);
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const size_t wbytes = ft_warp_bytes(P.max_block);
    unsigned char *ws = smem + al16f(P.tab_bytes) + warp * wbytes;
    const BlkShared sh = blk_carve(ws, P.max_block);
    float *sgw = (float *)(ws + al16f(blk_shared_bytes(P.max_block)));   // [sigma | gamma | alpha sigma][FT_W]
    double *red = (double *)(smem + al16f(P.tab_bytes) + (FT_NT / 32) * wbytes);
    constexpr int LPR = 32 / VT;                   // lanes per row
    const int grp = lane / LPR, li = lane % LPR;   // row group in the warp, lane in row
    const int v0 = li * VT;                        // first vector of this lane
    const unsigned nw = gridDim.x * (FT_NT / 32), gw = blockIdx.x * (FT_NT / 32) + warp;
    const FtRange rg = d.wr[gw];
    const unsigned long long LIMIT = F.barrier_ns;
    __syncthreads();

    for (int j = 0; j < F.steps; ++j) {
        const float *qc = (j & 1) ? d.q1 : d.q0;
        float *qp = (j & 1) ? d.q0 : d.q1;
        // ---------------- phase A: products ----------------
        // chunk c of ck_rows rows goes to warp c mod W, so all warps sweep the rows together
        // and the targets of nearby exchanges are still in L2; a warp's partial for sector s
        // sums its chunks of s and goes to parta[s][warp]
        {
            ef::df dot[VT];
#pragma unroll
            for (int q = 0; q < VT; ++q) dot[q] = ef::df{0.0f, 0.0f};
            int curA = -1;
            bool act = false;
            for (uint32_t c = gw; c < F.nchunks; c += nw) {
                int A = curA < 0 ? 0 : curA;
                while (d.ck_cs[A + 1] <= c) ++A;
                const uint64_t g0 = d.rowoff[A] + (uint64_t)(c - d.ck_cs[A]) * F.ck_rows;
                const uint64_t g1 = g0 + F.ck_rows < d.rowoff[A + 1] ? g0 + F.ck_rows : d.rowoff[A + 1];
                if (A != curA) {
                    if (curA >= 0) ft_warp_flush<VT>(dot, d.parta, (uint32_t)curA * nw + gw, lane, grp, v0);
                    curA = A;
                    act = d.sec_active[A] != 0;
                    __syncwarp();
                    if (act) {
                        const int sv = A * FT_W + lane;
                        sgw[lane] = (float)d.sig_cur[sv];
                        sgw[FT_W + lane] = (float)(d.beta_prev[sv] * d.sig_prev[sv]);
                    }
                }
                if (!act) continue;
                const uint64_t base = d.rowoff[A];
                for (uint32_t it = d.ck_it0[c]; it < (uint32_t)F.nitems; ++it) {
                    const uint32_t item = d.items[it];
                    if ((int)(item >> 16) != A) break;     // the chunk ends at the sector's end
                    const uint32_t h = item & 0xFFFFu;
                    const int k = A - __popc(h);
                    const uint32_t off = blk_off(P, tb, h, k);
                    const uint32_t n = tb.C[P.K * (P.A + 1) + k];
                    const uint64_t ig0 = base + off;
                    if (ig0 >= g1) break;
                    const uint32_t ra = ig0 < g0 ? (uint32_t)(g0 - ig0) : 0u;
                    const uint32_t rb = ig0 + n > g1 ? (uint32_t)(g1 - ig0) : n;
                    __syncwarp();                  // the previous block's lists are read no more
                    ft_warp_setup(P, tb, h, k, off, sh, lane);
                    __syncwarp();
                    const float *Xb = qc + ig0 * FT_W + v0;   // the block's rows, this lane's vectors
                    const uint16_t *Uk = tb.U + k * P.nb1;
                    const uint16_t *lw = P.lw + P.lwoff[k];
                    for (uint32_t r = ra + grp; r < rb; r += VT) {
                        const uint32_t l = __ldg(lw + r);
                        float acc[NC][VT];
                        int cnt[NC];
#pragma unroll
                        for (int cl = 0; cl < NC; ++cl) {
                            float *ac = acc[cl];
#pragma unroll
                            for (int q = 0; q < VT; ++q) ac[q] = 0.0f;
                            int mc = blk_low_hops(P, tb, cl, l, r, Uk, [&](uint32_t r2) {
                                float xv[VT];
                                ft_ld<VT>(Xb + (size_t)r2 * FT_W, xv);
#pragma unroll
                                for (int q = 0; q < VT; ++q) ac[q] += xv[q];
                            });
                            mc += blk_cross_hops(P, tb, cl, l, sh, [&](uint32_t jj) {
                                float xv[VT];
                                ft_ld<VT>(qc + (base + jj) * FT_W + v0, xv);
#pragma unroll
                                for (int q = 0; q < VT; ++q) ac[q] += xv[q];
                            });
                            // high exchanges: four independent gathers in flight (the far ones miss L2)
                            const int e1 = sh.hcs[cl + 1];
                            int e = sh.hcs[cl];
                            for (; e + 4 <= e1; e += 4) {
                                float x0[VT], x1[VT], x2[VT], x3[VT];
                                ft_ld<VT>(Xb + (int64_t)((int64_t)r + sh.hcd[e]) * FT_W, x0);
                                ft_ld<VT>(Xb + (int64_t)((int64_t)r + sh.hcd[e + 1]) * FT_W, x1);
                                ft_ld<VT>(Xb + (int64_t)((int64_t)r + sh.hcd[e + 2]) * FT_W, x2);
                                ft_ld<VT>(Xb + (int64_t)((int64_t)r + sh.hcd[e + 3]) * FT_W, x3);
#pragma unroll
                                for (int q = 0; q < VT; ++q) ac[q] += (x0[q] + x1[q]) + (x2[q] + x3[q]);
                            }
                            for (; e < e1; ++e) {
                                float xv[VT];
                                ft_ld<VT>(Xb + (int64_t)((int64_t)r + sh.hcd[e]) * FT_W, xv);
#pragma unroll
                                for (int q = 0; q < VT; ++q) ac[q] += xv[q];
                            }
                            cnt[cl] = mc + (sh.hcs[cl + 1] - sh.hcs[cl]);
                        }
                        const uint64_t row = ig0 + r;
                        float xov[VT];
                        ft_ld<VT>(Xb + (size_t)r * FT_W, xov);
#pragma unroll
                        for (int q = 0; q < VT; ++q) {
                            const float xo = xov[q];
                            float y = 0.0f;
#pragma unroll
                            for (int cl = 0; cl < NC; ++cl)
                                y += P.gq[cl] * (2.0f * acc[cl][q] + (float)(P.ntot[cl] - 2 * cnt[cl]) * xo);
                            const float u = sgw[v0 + q] * y - sgw[FT_W + v0 + q] * qp[row * FT_W + v0 + q];
                            qp[row * FT_W + v0 + q] = u;
                            dot[q] = ef::df_add(dot[q], ef::two_prod(sgw[v0 + q] * xo, u));
                        }
                    }
                }
            }
            if (curA >= 0) ft_warp_flush<VT>(dot, d.parta, (uint32_t)curA * nw + gw, lane, grp, v0);
            // the CTA's warp partials, summed in warp order (written by this CTA just now)
            __syncthreads();
            const unsigned w0 = blockIdx.x * (FT_NT / 32);
            for (int t = threadIdx.x; t < F.nsec * FT_W; t += FT_NT) {
                const int s = t / FT_W, v = t % FT_W;
                const double *ps = d.parta + ((size_t)s * nw + w0) * FT_W + v;
                double a = 0.0;
#pragma unroll
                for (int i = 0; i < FT_NT / 32; ++i) a += ps[(size_t)i * FT_W];
                d.partc[((size_t)s * F.nctas + blockIdx.x) * FT_W + v] = a;
            }
        }
        if (!grid_sync(d.bar, F.nctas, LIMIT)) return;
        // ---------------- phase B: alpha ----------------
        ft_sector_sums_a(F, red, [&](int s, int v, double a) {
            const int t = s * FT_W + v;
            if (d.done[t]) return;
            d.alpha[(size_t)t * F.steps + j] = a;
            d.scale[t] = fmax(d.scale[t], fabs(a));
            d.as[t] = a * d.sig_cur[t];
        });
        if (!grid_sync(d.bar, F.nctas, LIMIT)) return;
        // ---------------- phase C: update (a stream over the warp's rows) ----------------
        // lane: float4 number lane % 8 of a row, i.e. vectors 4 (lane % 8) .. + 3; the four
        // lanes of one float4 position are row groups 0..3 (ft_warp_flush<4> layout)
        if (rg.g0 < rg.g1) {
            ef::df nn[4];
#pragma unroll
            for (int q = 0; q < 4; ++q) nn[q] = ef::df{0.0f, 0.0f};
            const int c4 = lane & 7, g4 = lane >> 3;
            int A = ft_sector_of(d, F.nsec, rg.g0);
            uint32_t slot = rg.slot0;
            for (;; ++A, ++slot) {
                const uint64_t a0 = rg.g0 > d.rowoff[A] ? rg.g0 : d.rowoff[A];
                const uint64_t a1 = rg.g1 < d.rowoff[A + 1] ? rg.g1 : d.rowoff[A + 1];
                if (d.sec_active[A]) {
                    __syncwarp();
                    sgw[2 * FT_W + lane] = (float)d.as[A * FT_W + lane];
                    __syncwarp();
                    float as4[4];
#pragma unroll
                    for (int q = 0; q < 4; ++q) as4[q] = sgw[2 * FT_W + 4 * c4 + q];
                    for (uint64_t row = a0 + g4; row < a1; row += 4) {
                        const size_t ix = row * FT_W + 4 * c4;
                        const float4 u = *(const float4 *)(qp + ix);
                        const float4 x = __ldcs((const float4 *)(qc + ix));
                        float4 w;
                        w.x = u.x - as4[0] * x.x; w.y = u.y - as4[1] * x.y;
                        w.z = u.z - as4[2] * x.z; w.w = u.w - as4[3] * x.w;
                        *(float4 *)(qp + ix) = w;
                        nn[0] = ef::df_add(nn[0], ef::two_prod(w.x, w.x));
                        nn[1] = ef::df_add(nn[1], ef::two_prod(w.y, w.y));
                        nn[2] = ef::df_add(nn[2], ef::two_prod(w.z, w.z));
                        nn[3] = ef::df_add(nn[3], ef::two_prod(w.w, w.w));
                    }
                }
                ft_warp_flush<4>(nn, d.part, slot, lane, g4, 4 * c4);
                if (a1 >= rg.g1) break;
            }
        }
        if (!grid_sync(d.bar, F.nctas, LIMIT)) return;
        // ---------------- phase D: beta ----------------
        ft_sector_sums(F, red, [&](int s, int v, double sum) {
            const int t = s * FT_W + v;
            bool act = false;
            if (!d.done[t]) {
                const double b = sqrt(sum);
                d.beta[(size_t)t * F.steps + j] = b;
                d.nsteps[t] = j + 1;
                // stop when beta is at the noise floor or the sector is exhausted
                if (b <= FT_TOL * d.scale[t] || (uint32_t)(j + 1) >= d.secdim[s]) {
                    d.done[t] = 1;
                    d.sig_cur[t] = 0.0;
                    d.sig_prev[t] = 0.0;
                    d.beta_prev[t] = 0.0;
                    d.as[t] = 0.0;
                } else {
                    d.scale[t] = fmax(d.scale[t], b);
                    d.sig_prev[t] = d.sig_cur[t];
                    d.sig_cur[t] = 1.0 / b;
                    d.beta_prev[t] = b;
                    act = true;
                }
            }
            // a sector stays active while any of its vectors runs (warp 0 holds one sector)
            const unsigned any = __ballot_sync(0xffffffffu, act);
            if (v == 0) d.sec_active[s] = any != 0u;
        });
        if (!grid_sync(d.bar, F.nctas, LIMIT)) return;
    }
}

// ---- tridiagonal eigen-decomposition with the first components -------------------------
// Implicit symmetric QR with Wilkinson shifts (Golub and Van Loan, Sec. 8.3): each sweep
// chases a bulge down the unreduced block with Givens rotations; the rotations are also
// applied to z, the first row of the accumulated eigenvector matrix.
__device__ void tri_ql_first(int m, double *dg, double *e, double *z) {
    for (int i = 0; i < m; ++i) z[i] = i == 0 ? 1.0 : 0.0;
    int hi = m - 1, guard = 0;
    while (hi > 0 && guard < 60 * m) {
        const double tol = 2.220446049250313e-16 * (fabs(dg[hi - 1]) + fabs(dg[hi]));
        if (fabs(e[hi - 1]) <= tol) { e[hi - 1] = 0.0; --hi; continue; }
        int lo = hi - 1;
        while (lo > 0 && fabs(e[lo - 1]) > 2.220446049250313e-16 * (fabs(dg[lo - 1]) + fabs(dg[lo]))) --lo;
        ++guard;
        // Wilkinson shift: eigenvalue of the trailing 2x2 block closer to dg[hi]
        const double dd = 0.5 * (dg[hi - 1] - dg[hi]);
        const double eh = e[hi - 1];
        const double den = dd + copysign(sqrt(dd * dd + eh * eh), dd == 0.0 ? 1.0 : dd);
        const double mu = dg[hi] - eh * eh / den;
        double x = dg[lo] - mu, y = e[lo];
        for (int kk = lo; kk < hi; ++kk) {
            const double r = hypot(x, y);
            const double c = r == 0.0 ? 1.0 : x / r, s = r == 0.0 ? 0.0 : y / r;
            if (kk > lo) e[kk - 1] = r;
            const double a = dg[kk], b = e[kk], cc = dg[kk + 1];
            dg[kk] = c * c * a + 2.0 * c * s * b + s * s * cc;
            dg[kk + 1] = s * s * a - 2.0 * c * s * b + c * c * cc;
            e[kk] = c * s * (cc - a) + (c * c - s * s) * b;
            const double zk = z[kk], zk1 = z[kk + 1];
            z[kk] = c * zk + s * zk1;
            z[kk + 1] = -s * zk + c * zk1;
            if (kk + 1 < hi) {
                x = e[kk];
                y = s * e[kk + 1];
                e[kk + 1] = c * e[kk + 1];
            }
        }
    }
}

__global__ void k_ft_eig(FtParams F, double *scratch) {
    const FtDev &d = F.d;
    const int t = blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= F.nsec * FT_W) return;
    const int v = t % FT_W;
    if ((F.exact_mask >> (t / FT_W)) & 1ull) return;   // filled by k_ft_exact
    const int m = (v < F.R) ? d.nsteps[t] : 0;
    d.mlen[t] = m;
    if (m == 0) return;
    double *dg = scratch + (size_t)t * 3 * F.steps, *e = dg + F.steps, *z = e + F.steps;
    for (int i = 0; i < m; ++i) dg[i] = d.alpha[(size_t)t * F.steps + i];
    for (int i = 0; i + 1 < m; ++i) e[i] = d.beta[(size_t)t * F.steps + i];
    if (m > 1) e[m - 1] = 0.0;
    tri_ql_first(m, dg, e, z);
    for (int i = 0; i < m; ++i) {
        d.theta[(size_t)t * F.steps + i] = dg[i];
        d.tau[(size_t)t * F.steps + i] = z[i] * z[i];
    }
}

// Dense H of one small sector (rows by the paper's decode/encode, Eq. E-4-b), its
// eigen-decomposition by parallel cyclic Jacobi (Brent-Luk round-robin ordering of the
// rotations, each zeroing one off-diagonal pair as in Golub and Van Loan, Sec. 8.5),
// then theta_k = E_k and tau_k = <r^|psi_k>^2 for every start vector r^ = r / |r|.
__global__ void __launch_bounds__(256) k_ft_exact(FtParams F, BondParams bp, const uint32_t *__restrict__ cdall,
                                                  double *__restrict__ mats) {
    const FtDev &d = F.d;
    const ExactSec ex = F.ex[blockIdx.x];
    const int n = ex.dim;
    double *H = mats + ex.mat_off, *V = H + (size_t)n * n;
    __shared__ int sp[256], sq[256];
    __shared__ double sc[256], ss[256], red[8];
    __shared__ int s_stop;
    for (int t = threadIdx.x; t < n * n; t += blockDim.x) {
        H[t] = 0.0;
        V[t] = (t / n == t % n) ? 1.0 : 0.0;
    }
    __syncthreads();
    Codec<uint32_t> c{cdall + ex.cd_off, F.P.N, 1, ex.A, 1, 3, ex.cd_rowlen};
    for (int i = threadIdx.x; i < n; i += blockDim.x) {
        const uint64_t w = c.decode((uint32_t)i);
        double dg = 0.0;
        for (int t = 0; t < bp.nb; ++t) {
            const int p = bp.p[t], q = bp.q[t];
            const int ap = dig(w, p, 1), aq = dig(w, q, 1);
            dg += bp.jm[t] * (0.5 - ap) * (0.5 - aq);
            if (ap != aq) {
                const uint32_t j = (uint32_t)i + c.delta(w, p, q, ap ? -1 : +1);
                H[(size_t)i * n + j] += bp.jm[t] * 0.5;
            }
        }
        H[(size_t)i * n + i] += dg;
    }
    __syncthreads();
    const int m = n + (n & 1);            // players of the round-robin (one dummy if n is odd)
    for (int sweep = 0; sweep < 40 && n > 1; ++sweep) {
        // stop when the off-diagonal part is negligible
        double off = 0.0, tot = 0.0;
        for (int t = threadIdx.x; t < n * n; t += blockDim.x) {
            const double h = H[t];
            tot += h * h;
            if (t / n != t % n) off += h * h;
        }
        off = block_sum<256>(off, red);
        __syncthreads();
        tot = block_sum<256>(tot, red);
        if (threadIdx.x == 0) s_stop = off <= 1e-30 * tot;
        __syncthreads();
        if (s_stop) break;
        for (int round = 0; round < m - 1; ++round) {
            for (int k = threadIdx.x; k < m / 2; k += blockDim.x) {
                int p, q;
                if (k == 0) { p = m - 1; q = round; }
                else { p = (round + k) % (m - 1); q = (round - k + (m - 1)) % (m - 1); }
                if (p > q) { const int tt = p; p = q; q = tt; }
                double cc = 1.0, sn = 0.0;
                if (q < n) {
                    const double apq = H[(size_t)p * n + q];
                    if (apq != 0.0) {
                        const double tau = (H[(size_t)q * n + q] - H[(size_t)p * n + p]) / (2.0 * apq);
                        const double t = (tau >= 0.0 ? 1.0 : -1.0) / (fabs(tau) + sqrt(1.0 + tau * tau));
                        cc = 1.0 / sqrt(1.0 + t * t);
                        sn = t * cc;
                    }
                }
                sp[k] = p; sq[k] = q; sc[k] = cc; ss[k] = sn;
            }
            __syncthreads();
            for (int t = threadIdx.x; t < (m / 2) * n; t += blockDim.x) {   // rows: A <- J^T A
                const int k = t / n, j = t % n;
                if (sq[k] >= n) continue;
                const double a = H[(size_t)sp[k] * n + j], b = H[(size_t)sq[k] * n + j];
                H[(size_t)sp[k] * n + j] = sc[k] * a - ss[k] * b;
                H[(size_t)sq[k] * n + j] = ss[k] * a + sc[k] * b;
            }
            __syncthreads();
            for (int t = threadIdx.x; t < (m / 2) * n; t += blockDim.x) {   // columns: A <- A J, V <- V J
                const int k = t / n, i = t % n;
                if (sq[k] >= n) continue;
                const double a = H[(size_t)i * n + sp[k]], b = H[(size_t)i * n + sq[k]];
                H[(size_t)i * n + sp[k]] = sc[k] * a - ss[k] * b;
                H[(size_t)i * n + sq[k]] = ss[k] * a + sc[k] * b;
                const double va = V[(size_t)i * n + sp[k]], vb = V[(size_t)i * n + sq[k]];
                V[(size_t)i * n + sp[k]] = sc[k] * va - ss[k] * vb;
                V[(size_t)i * n + sq[k]] = ss[k] * va + sc[k] * vb;
            }
            __syncthreads();
        }
    }
    // weights of every start vector
    const double inv = 1.0 / sqrt((double)n);
    for (int t = threadIdx.x; t < F.R * n; t += blockDim.x) {
        const int r = t / n, kk = t % n;
        const uint64_t stream = sm64(F.seed, ((uint64_t)ex.A << 20) + (uint64_t)r);
        double o = 0.0;
        for (int i = 0; i < n; ++i) o += V[(size_t)i * n + kk] * ((sm64(stream, (uint64_t)i) >> 63) ? -inv : inv);
        const size_t sv = (size_t)ex.A * FT_W + r;
        d.theta[sv * F.steps + kk] = H[(size_t)kk * n + kk];
        d.tau[sv * F.steps + kk] = o * o;
    }
    for (int r = threadIdx.x; r < FT_W; r += blockDim.x) d.mlen[(size_t)ex.A * FT_W + r] = r < F.R ? n : 0;
}

// one block: e_ref = min theta, then Z and E sums for each temperature (fixed order)
__global__ void k_ft_thermo(FtParams F, const double *temps, int n_t) {
    const FtDev &d = F.d;
    __shared__ double red[32];
    __shared__ double s_ref;
    const int nst = F.nsec * FT_W;
    double mn = 1e308;
    for (int t = threadIdx.x; t < nst; t += blockDim.x)
        for (int i = 0; i < d.mlen[t]; ++i) mn = fmin(mn, d.theta[(size_t)t * F.steps + i]);
    for (int o = 16; o > 0; o >>= 1) mn = fmin(mn, __shfl_down_sync(0xffffffffu, mn, o));
    if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = mn;
    __syncthreads();
    if (threadIdx.x == 0) {
        double m = 1e308;
        for (int w = 0; w < (int)(blockDim.x >> 5); ++w) m = fmin(m, red[w]);
        s_ref = m;
        *d.eref = m;
    }
    __syncthreads();
    const double e_ref = s_ref;
    for (int it = 0; it < n_t; ++it) {
        const double T = temps[it];
        double z = 0.0, ez = 0.0;
        for (int t = threadIdx.x; t < nst; t += blockDim.x) {
            const int s = t / FT_W;
            const double wgt = (double)d.secdim[s] / (double)F.R;
            for (int i = 0; i < d.mlen[t]; ++i) {
                const double th = d.theta[(size_t)t * F.steps + i];
                const double b = d.tau[(size_t)t * F.steps + i] * exp(-(th - e_ref) / T) * wgt;
                z += b;
                ez += b * th;
            }
        }
        __syncthreads();
        double zs = block_sum<1024>(z, red);
        __syncthreads();
        double es = block_sum<1024>(ez, red);
        if (threadIdx.x == 0) { d.zsum[it] = zs; d.esum[it] = es / zs; }
        __syncthreads();
    }
}

// ---- host --------------------------------------------------------------------------------
struct FtLayout {
    size_t q0, q1, st, ab, part, wr, slo, parta, partc, ckit, ckcs, sec, bar, items, rowoff, secdim, theta, tau, mlen, therm, temps, eigs,
        xcd, xmat, total;
};

static int ft_choose_K(int N) {
    // largest K (8..16, K <= N-2) whose biggest block of 32-float rows fits ~75 KB, so
    // two CTAs fit on an SM (K = 11: 462 rows, 59 KB)
    int best = -1;
    for (int K = 8; K <= 16 && K <= N - 2; ++K) {
        uint64_t c = 1;
        for (int i = 0; i < K / 2; ++i) c = c * (K - i) / (i + 1);
        if (c * FT_W * 4 <= 75 * 1024) best = K;
    }
    return best;
}

static FtLayout ft_layout(int N, int nsec, int R, int steps, int nitems, int nctas, int n_t, size_t xcd_words,
                          size_t xmat_doubles, size_t nchunks) {
    (void)R;
    FtLayout L{};
    auto a = [](size_t x) { return (x + 255) & ~(size_t)255; };
    const uint64_t rows = 1ull << N;     // sum of all sector dimensions for s = 1/2
    const size_t nst = (size_t)nsec * FT_W;
    size_t o = 0;
    L.q0 = o; o += a(rows * FT_W * 4);
    L.q1 = o; o += a(rows * FT_W * 4);
    L.st = o; o += a(nst * 8 * 5 + nst * 4 * 2);
    L.ab = o; o += a(nst * (size_t)steps * 8 * 2);
    const size_t nslots = (size_t)nctas * (FT_NT / 32) + nsec + 1;   // bound on the warp-sector pairs
    L.part = o; o += a(nslots * FT_W * 8);
    L.wr = o; o += a((size_t)nctas * (FT_NT / 32) * sizeof(FtRange));
    L.slo = o; o += a((size_t)(nsec + 1) * 4);
    L.parta = o; o += a((size_t)nsec * nctas * (FT_NT / 32) * FT_W * 8);
    L.partc = o; o += a((size_t)nsec * nctas * FT_W * 8);
    L.ckit = o; o += a((nchunks > 0 ? nchunks : 1) * 4);
    L.ckcs = o; o += a((size_t)(nsec + 1) * 4);
    L.sec = o; o += a(FT_MAXS * 4);
    L.bar = o; o += a(sizeof(GridBar));
    L.items = o; o += a((size_t)nitems * 4);
    L.rowoff = o; o += a((size_t)(nsec + 1) * 8);
    L.secdim = o; o += a((size_t)nsec * 4);
    L.theta = o; o += a(nst * (size_t)steps * 8);
    L.tau = o; o += a(nst * (size_t)steps * 8);
    L.mlen = o; o += a(nst * 4);
    L.therm = o; o += a((size_t)(2 * n_t + 1) * 8);
    L.temps = o; o += a((size_t)(n_t > 0 ? n_t : 1) * 8);
    L.eigs = o; o += a(nst * 3 * (size_t)steps * 8);
    L.xcd = o; o += a((xcd_words > 0 ? xcd_words : 1) * 4);
    L.xmat = o; o += a((xmat_doubles > 0 ? xmat_doubles : 1) * 8);
    L.total = o;
    return L;
}

template <int NC, int VT>
static const void *ft_kernel() { return (const void *)k_ftlm<NC, VT>; }

static const void *pick_kernel(int nc, int vt) {
    if (nc == 1) return vt == 1 ? ft_kernel<1, 1>() : vt == 2 ? ft_kernel<1, 2>() : ft_kernel<1, 4>();
    if (nc == 2) return vt == 1 ? ft_kernel<2, 1>() : vt == 2 ? ft_kernel<2, 2>() : ft_kernel<2, 4>();
    return vt == 1 ? ft_kernel<4, 1>() : vt == 2 ? ft_kernel<4, 2>() : ft_kernel<4, 4>();
}

static size_t ft_smem(const BlkParams &P, int nsec) {
    (void)nsec;
    size_t o = al16f(P.tab_bytes);
    o += (FT_NT / 32) * ft_warp_bytes(P.max_block);
    o += al16f((size_t)(FT_NT / FT_W) * FT_W * 8);    // sector-sum scratch
    return o;
}

// The warps' row ranges (equal shares of all 2^N rows) and their partial-sum slots.
// items: the blocks (A << 16 | h) in row order; C(K, k) rows each.
static void ft_ranges(int n_sites, int K, const hm_basis &full, const std::vector<uint32_t> &items, int W,
                      uint32_t ck_rows, std::vector<FtRange> *wr, std::vector<uint32_t> *slo,
                      std::vector<uint32_t> *ck_it0, std::vector<uint32_t> *ck_cs) {
    const int N = n_sites, nsec = N + 1, Wd = N + 1;
    std::vector<uint64_t> r0(items.size() + 1, 0);
    for (size_t i = 0; i < items.size(); ++i) {
        const int A = (int)(items[i] >> 16);
        const int k = A - __builtin_popcount(items[i] & 0xFFFFu);
        r0[i + 1] = r0[i] + full.D[(size_t)K * Wd + k];
    }
    std::vector<uint64_t> rowoff(nsec + 1, 0);
    for (int A = 0; A < nsec; ++A) rowoff[A + 1] = rowoff[A] + full.D[(size_t)N * Wd + A];
    const uint64_t T = r0.back();
    auto sector_of = [&](uint64_t g) { return (int)(std::upper_bound(rowoff.begin(), rowoff.end(), g) - rowoff.begin()) - 1; };
    wr->assign(W, FtRange{});
    std::vector<int> slot_sec;
    for (int w = 0; w < W; ++w) {
        FtRange &g = (*wr)[w];
        g.g0 = T * (uint64_t)w / (uint64_t)W;
        g.g1 = T * (uint64_t)(w + 1) / (uint64_t)W;
        g.slot0 = (uint32_t)slot_sec.size();
        if (g.g0 >= g.g1) { g.it0 = (uint32_t)items.size(); continue; }
        g.it0 = (uint32_t)(std::upper_bound(r0.begin(), r0.end(), g.g0) - r0.begin() - 1);
        for (int A = sector_of(g.g0); A <= sector_of(g.g1 - 1); ++A) slot_sec.push_back(A);
    }
    slo->assign(nsec + 1, 0);
    size_t i = 0;
    for (int s = 0; s <= nsec; ++s) {
        while (i < slot_sec.size() && slot_sec[i] < s) ++i;
        (*slo)[s] = (uint32_t)i;
    }
    // product-phase chunks: each sector cut into runs of ck_rows rows
    ck_it0->clear();
    ck_cs->assign(nsec + 1, 0);
    for (int A = 0; A < nsec; ++A) {
        (*ck_cs)[A] = (uint32_t)ck_it0->size();
        for (uint64_t g = rowoff[A]; g < rowoff[A + 1]; g += ck_rows)
            ck_it0->push_back((uint32_t)(std::upper_bound(r0.begin(), r0.end(), g) - r0.begin() - 1));
    }
    (*ck_cs)[nsec] = (uint32_t)ck_it0->size();
}

// rows per product-phase chunk: HM_FT_CHUNK (16..1024), default 64
static uint32_t ft_chunk_rows() {
    const char *e = getenv("HM_FT_CHUNK");
    const int v = e ? atoi(e) : 64;
    return (uint32_t)(v < 16 ? 16 : v > 1024 ? 1024 : v);
}

// how long a grid barrier of the persistent kernel waits before it gives up: 5 s, or
// HM_FT_BARRIER_NS (0 .. 5e9 ns; a test sets 0 to make the first wait give up)
static unsigned long long ft_barrier_ns() {
    const unsigned long long dflt = 5000000000ull;
    const char *e = getenv("HM_FT_BARRIER_NS");
    if (!e || !*e) return dflt;
    const long long v = atoll(e);
    return v < 0 ? 0ull : (unsigned long long)v > dflt ? dflt : (unsigned long long)v;
}

// vectors-per-lane tiling chosen by timing each candidate once per (N, bonds) shape
static std::map<std::pair<int, int>, int> g_ft_tuned;

struct FtSetup {
    hm_basis full;                   // tables with the full binomial table (A = N)
    FtParams F;
    BondParams bp;
    FtLayout L;
    size_t smem;
    int nctas;
    std::vector<uint32_t> xcd;       // CD tables of the exactly diagonalised sectors
    std::vector<FtRange> wr;         // per warp
    std::vector<uint32_t> slo;       // per sector, + 1
    std::vector<uint32_t> ck_it0;    // per product-phase chunk
    std::vector<uint32_t> ck_cs;     // per sector, + 1
};

static int ft_prepare(int n_sites, int two_s, int n_bonds, const int32_t *u, const int32_t *v,
                      const double *J, int R, int steps, int n_t, FtSetup *S, std::vector<uint32_t> *items) {
    if (two_s != 1) return fail(HM_EINVAL, "ftlm_run supports s = 1/2 (two_s = 1)");
    if (R < 1 || R > FT_W) return fail(HM_EINVAL, "R must be in 1..%d", FT_W);
    if (steps < 1 || steps > 2000) return fail(HM_EINVAL, "steps must be in 1..2000");
    if (n_t < 0 || n_t > 4096) return fail(HM_EINVAL, "n_t must be in 0..4096");
    const int K = ft_choose_K(n_sites);
    if (K < 0 || n_sites > 32) return fail(HM_EINVAL, "ftlm_run needs 10 <= n_sites <= 32");
    HM_TRY(build_tables(n_sites, 1, -n_sites, &S->full));      // A = N: full table
    BondParams &bp = S->bp;
    HM_TRY(make_bonds(&S->full, n_bonds, u, v, J, &bp));
    memset(&S->F, 0, sizeof S->F);
    const int prc = blk_plan(&S->full, bp, K, &S->F.P);
    if (prc < 0) return prc;
    if (prc > 0 || S->F.P.perbond)
        return fail(HM_EINVAL, "ftlm_run: more than %d coupling classes or %d bonds", HM_BLK_MAXC, HM_BLK_MAXB);
    // the plan's block size was taken for A = N; use the largest over all sectors
    uint64_t mb = 1;
    for (int i = 0; i < K / 2; ++i) mb = mb * (K - i) / (i + 1);
    S->F.P.max_block = (int)mb;
    const int nsec = n_sites + 1;
    items->clear();
    const int H = n_sites - K;
    for (int A = 0; A <= n_sites; ++A)
        for (uint32_t h = 0; h < (1u << H); ++h) {
            const int k = A - __builtin_popcount(h);
            if (k >= 0 && k <= K) items->push_back(((uint32_t)A << 16) | h);
        }
    S->F.nsec = nsec;
    S->F.R = R;
    S->F.steps = steps;
    // sectors of dimension <= steps (and <= 512): exact treatment
    S->xcd.clear();
    uint64_t xmat = 0;
    for (int A = 0; A <= n_sites; ++A) {
        const int W = n_sites + 1;
        const uint64_t dimA = S->full.D[(size_t)n_sites * W + A];
        if (dimA > (uint64_t)steps || dimA > 512) continue;
        if (S->F.nexact == FT_MAXEXACT) return fail(HM_EINVAL, "ftlm_run: too many small sectors");
        hm_basis sb;
        HM_TRY(build_tables(n_sites, 1, n_sites - 2 * A, &sb));
        ExactSec &ex = S->F.ex[S->F.nexact++];
        ex.A = A;
        ex.dim = (int)dimA;
        ex.cd_off = (uint32_t)S->xcd.size();
        ex.cd_rowlen = sb.view.cd_rowlen;
        ex.cd_len = sb.view.cd_len;
        for (int k = 0; k < sb.view.cd_len; ++k) S->xcd.push_back((uint32_t)sb.cd[k]);
        ex.mat_off = xmat;
        xmat += 2 * dimA * dimA;
        S->F.exact_mask |= 1ull << A;
    }
    S->F.nitems = (int)items->size();
    S->smem = ft_smem(S->F.P, nsec);
    if (S->smem > 227 * 1024) return fail(HM_EINVAL, "ftlm_run: shared memory plan too large");
    // co-resident CTAs per SM: the fewest any tiling allows (at most FT_CTAS)
    int per_sm = FT_CTAS;
    for (int vt : {1, 2, 4}) {
        const void *kfn = pick_kernel(S->F.P.nc, vt);
        int p = 0;
        HM_CUDA(raise_smem_limit(kfn, (int)S->smem));
        HM_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&p, kfn, FT_NT, S->smem));
        per_sm = std::min(per_sm, p);
    }
    if (per_sm < 1) return fail(HM_EINVAL, "ftlm_run: kernel does not fit on an SM");
    S->nctas = sm_count() * per_sm;   // cooperative: all resident
    S->F.nctas = (unsigned)S->nctas;
    S->F.ck_rows = ft_chunk_rows();
    ft_ranges(n_sites, K, S->full, *items, S->nctas * (FT_NT / 32), S->F.ck_rows, &S->wr, &S->slo, &S->ck_it0,
              &S->ck_cs);
    S->F.nchunks = (uint32_t)S->ck_it0.size();
    S->L = ft_layout(n_sites, nsec, R, steps, S->F.nitems, S->nctas, n_t, S->xcd.size(), (size_t)xmat,
                     S->F.nchunks);
    return HM_OK;
}

static void ft_bind(FtSetup *S, unsigned char *w) {
    const FtLayout &L = S->L;
    FtDev &d = S->F.d;
    const size_t nst = (size_t)S->F.nsec * FT_W;
    d.q0 = (float *)(w + L.q0);
    d.q1 = (float *)(w + L.q1);
    double *st = (double *)(w + L.st);
    d.sig_cur = st; d.sig_prev = st + nst; d.beta_prev = st + 2 * nst; d.scale = st + 3 * nst; d.as = st + 4 * nst;
    d.done = (int *)(st + 5 * nst);
    d.nsteps = d.done + nst;
    d.alpha = (double *)(w + L.ab);
    d.beta = d.alpha + nst * S->F.steps;
    d.part = (double *)(w + L.part);
    d.wr = (const FtRange *)(w + L.wr);
    d.slo = (const uint32_t *)(w + L.slo);
    d.parta = (double *)(w + L.parta);
    d.partc = (double *)(w + L.partc);
    d.ck_it0 = (const uint32_t *)(w + L.ckit);
    d.ck_cs = (const uint32_t *)(w + L.ckcs);
    d.sec_active = (int *)(w + L.sec);
    d.bar = (GridBar *)(w + L.bar);
    d.items = (const uint32_t *)(w + L.items);
    d.rowoff = (const uint64_t *)(w + L.rowoff);
    d.secdim = (const uint32_t *)(w + L.secdim);
    d.theta = (double *)(w + L.theta);
    d.tau = (double *)(w + L.tau);
    d.mlen = (int *)(w + L.mlen);
    double *th = (double *)(w + L.therm);
    d.zsum = th;
    d.esum = th + 1;   // reassigned with n_t below
    d.eref = th;
}

static int ft_launch_persistent(FtSetup *S, int vt, cudaStream_t st) {
    const void *kfn = pick_kernel(S->F.P.nc, vt);
    HM_CUDA(raise_smem_limit(kfn, (int)S->smem));
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3(S->nctas);
    cfg.blockDim = dim3(FT_NT);
    cfg.dynamicSmemBytes = S->smem;
    cfg.stream = st;
    cudaLaunchAttribute at[1];
    at[0].id = cudaLaunchAttributeCooperative;
    at[0].val.cooperative = 1;
    cfg.attrs = at;
    cfg.numAttrs = 1;
    void *args[] = {(void *)&S->F};
    HM_CUDA(cudaLaunchKernelExC(&cfg, kfn, args));
    return HM_OK;
}

}  // namespace hm

using namespace hm;

extern "C" {

int ftlm_workspace(int n_sites, int two_s, int n_bonds, const int32_t *u, const int32_t *v,
                   const double *J, int R, int steps, int n_t, size_t *bytes) {
    if (!bytes) return fail(HM_EINVAL, "bytes is NULL");
    FtSetup S;
    std::vector<uint32_t> items;
    HM_TRY(ft_prepare(n_sites, two_s, n_bonds, u, v, J, R, steps, n_t, &S, &items));
    *bytes = S.L.total;
    return HM_OK;
}

int ftlm_run(int n_sites, int two_s, int n_bonds, const int32_t *u, const int32_t *v, const double *J,
             int R, int steps, uint64_t seed, const double *temps, int n_t, double *Z, double *E,
             double *e_ref, double *theta, double *tau, int *mlen, int vt, void *work,
             size_t work_bytes, void *stream) {
    if (n_t > 0 && (!temps || !Z || !E)) return fail(HM_EINVAL, "temperature arrays are NULL");
    if (vt != 0 && vt != 1 && vt != 2 && vt != 4) return fail(HM_EINVAL, "vt must be 0 (autotune), 1, 2 or 4");
    FtSetup S;
    std::vector<uint32_t> items;
    HM_TRY(ft_prepare(n_sites, two_s, n_bonds, u, v, J, R, steps, n_t, &S, &items));
    if (!work || work_bytes < S.L.total || ((uintptr_t)work & 255))
        return fail(HM_EWORKSPACE, "ftlm_run needs %zu workspace bytes (256-byte aligned)", S.L.total);
    cudaStream_t st = as_stream(stream);
    unsigned char *w = (unsigned char *)work;
    ft_bind(&S, w);
    S.F.seed = seed;
    S.F.barrier_ns = ft_barrier_ns();
    double *therm = (double *)(w + S.L.therm);
    S.F.d.eref = therm;
    S.F.d.zsum = therm + 1;
    S.F.d.esum = therm + 1 + n_t;
    // host-built inputs: items, sector row offsets and dimensions
    const int nsec = S.F.nsec;
    std::vector<uint64_t> rowoff(nsec + 1, 0);
    std::vector<uint32_t> dims(nsec);
    {
        const int W = S.full.view.S2 * n_sites + 1;
        for (int A = 0; A < nsec; ++A) {
            dims[A] = (uint32_t)S.full.D[(size_t)n_sites * W + A];
            rowoff[A + 1] = rowoff[A] + dims[A];
        }
    }
    HM_CUDA(cudaMemcpyAsync(w + S.L.items, items.data(), items.size() * 4, cudaMemcpyHostToDevice, st));
    HM_CUDA(cudaMemcpyAsync(w + S.L.rowoff, rowoff.data(), rowoff.size() * 8, cudaMemcpyHostToDevice, st));
    HM_CUDA(cudaMemcpyAsync(w + S.L.secdim, dims.data(), dims.size() * 4, cudaMemcpyHostToDevice, st));
    HM_CUDA(cudaMemcpyAsync(w + S.L.wr, S.wr.data(), S.wr.size() * sizeof(FtRange), cudaMemcpyHostToDevice, st));
    HM_CUDA(cudaMemcpyAsync(w + S.L.slo, S.slo.data(), S.slo.size() * 4, cudaMemcpyHostToDevice, st));
    if (!S.ck_it0.empty())
        HM_CUDA(cudaMemcpyAsync(w + S.L.ckit, S.ck_it0.data(), S.ck_it0.size() * 4, cudaMemcpyHostToDevice, st));
    HM_CUDA(cudaMemcpyAsync(w + S.L.ckcs, S.ck_cs.data(), S.ck_cs.size() * 4, cudaMemcpyHostToDevice, st));
    if (!S.xcd.empty())
        HM_CUDA(cudaMemcpyAsync(w + S.L.xcd, S.xcd.data(), S.xcd.size() * 4, cudaMemcpyHostToDevice, st));
    double *d_temps = (double *)(w + S.L.temps);
    if (n_t > 0) HM_CUDA(cudaMemcpyAsync(d_temps, temps, n_t * 8, cudaMemcpyHostToDevice, st));
    // autotune the vectors-per-lane tiling on a short run (2 steps), once per shape
    int use_vt = vt;
    if (use_vt == 0) {
        auto key = std::make_pair(n_sites, S.F.P.nc * 1000 + S.F.P.nhb * 10 + R);
        auto it = g_ft_tuned.find(key);
        if (it != g_ft_tuned.end()) {
            use_vt = it->second;
        } else {
            float best = 1e30f;
            int bvt = 1;
            FtParams keep = S.F;
            S.F.steps = std::min(steps, 2);
            cudaEvent_t e0, e1;
            HM_CUDA(cudaEventCreate(&e0));
            HM_CUDA(cudaEventCreate(&e1));
            for (int cand : {1, 2, 4}) {
                k_ft_init<<<sm_count() * 4, 256, 0, st>>>(S.F);
                HM_CUDA(cudaGetLastError());
                HM_CUDA(cudaEventRecord(e0, st));
                HM_TRY(ft_launch_persistent(&S, cand, st));
                HM_CUDA(cudaEventRecord(e1, st));
                HM_CUDA(cudaEventSynchronize(e1));
                float ms = 0.0f;
                HM_CUDA(cudaEventElapsedTime(&ms, e0, e1));
                if (ms < best) { best = ms; bvt = cand; }
            }
            cudaEventDestroy(e0);
            cudaEventDestroy(e1);
            S.F = keep;
            use_vt = bvt;
            g_ft_tuned[key] = bvt;
        }
    }
    // the run: init, persistent steps, eigen-decompositions, sums -- one captured graph
    cudaStream_t cap;
    HM_CUDA(cudaStreamCreateWithFlags(&cap, cudaStreamNonBlocking));
    cudaGraph_t g = nullptr;
    cudaGraphExec_t ge = nullptr;
    int rc = HM_OK;
    cudaError_t e = cudaStreamBeginCapture(cap, cudaStreamCaptureModeThreadLocal);
    if (e != cudaSuccess) rc = cuda_fail(e, "ftlm capture");
    if (rc == HM_OK) {
        k_ft_init<<<sm_count() * 4, 256, 0, cap>>>(S.F);
        if ((e = cudaGetLastError()) != cudaSuccess) rc = cuda_fail(e, "k_ft_init");
        if (rc == HM_OK) rc = ft_launch_persistent(&S, use_vt, cap);
        if (rc == HM_OK) {
            const int nst = nsec * FT_W;
            k_ft_eig<<<(nst + 127) / 128, 128, 0, cap>>>(S.F, (double *)(w + S.L.eigs));
            if ((e = cudaGetLastError()) != cudaSuccess) rc = cuda_fail(e, "k_ft_eig");
            if (rc == HM_OK && S.F.nexact > 0) {
                k_ft_exact<<<S.F.nexact, 256, 0, cap>>>(S.F, S.bp, (const uint32_t *)(w + S.L.xcd),
                                                        (double *)(w + S.L.xmat));
                if ((e = cudaGetLastError()) != cudaSuccess) rc = cuda_fail(e, "k_ft_exact");
            }
        }
        cudaError_t e2 = cudaStreamEndCapture(cap, &g);
        if (rc == HM_OK && e2 != cudaSuccess) rc = cuda_fail(e2, "ftlm end capture");
    }
    if (rc == HM_OK && (e = cudaGraphInstantiate(&ge, g, 0)) != cudaSuccess) rc = cuda_fail(e, "ftlm instantiate");
    if (rc == HM_OK && (e = cudaGraphLaunch(ge, st)) != cudaSuccess) rc = cuda_fail(e, "ftlm graph launch");
    if (ge) cudaGraphExecDestroy(ge);
    if (g) cudaGraphDestroy(g);
    cudaStreamDestroy(cap);
    HM_TRY(rc);
    if (n_t > 0) {
        k_ft_thermo<<<1, 1024, 0, st>>>(S.F, d_temps, n_t);
        HM_CUDA(cudaGetLastError());
    }
    GridBar bar;
    HM_CUDA(cudaMemcpyAsync(&bar, S.F.d.bar, sizeof bar, cudaMemcpyDeviceToHost, st));
    std::vector<double> th(1 + 2 * (size_t)n_t);
    HM_CUDA(cudaMemcpyAsync(th.data(), therm, th.size() * 8, cudaMemcpyDeviceToHost, st));
    HM_CUDA(cudaStreamSynchronize(st));
    if (bar.abort) return fail(HM_ETIMEOUT, "ftlm_run: a grid barrier timed out");
    if (e_ref) *e_ref = th[0];
    for (int i = 0; i < n_t; ++i) { Z[i] = th[1 + i]; E[i] = th[1 + n_t + i]; }
    const size_t nst = (size_t)nsec * FT_W;
    if (theta) HM_CUDA(cudaMemcpy(theta, S.F.d.theta, nst * steps * 8, cudaMemcpyDeviceToHost));
    if (tau) HM_CUDA(cudaMemcpy(tau, S.F.d.tau, nst * steps * 8, cudaMemcpyDeviceToHost));
    if (mlen) HM_CUDA(cudaMemcpy(mlen, S.F.d.mlen, nst * 4, cudaMemcpyDeviceToHost));
    return use_vt;   // > 0: the tiling that ran (informational)
}

}  // extern "C"
