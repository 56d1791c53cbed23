// blk.cu -- host planning and the matvec kernel of the s = 1/2 block path (blk.cuh).
#include <algorithm>
#include <climits>
#include <cstdlib>
#include <cstring>
#include <cmath>
#include <map>
#include <tuple>
#include <type_traits>

#include "blk.cuh"
#include "blk_sweep.cuh"

namespace hm {


// ---------------------------------------------------------------------------------------
// tables (cached per basis and K)
// ---------------------------------------------------------------------------------------
// U[k][b1], R0[b0] and C[p][c] of blk.cuh from the D table of Eq. (E-3-c)
int blk_host_tables(const hm_basis *b, int K, std::vector<uint16_t> &U, std::vector<uint8_t> &R0,
                    std::vector<uint32_t> &C) {
    const SectorView &sv = b->view;
    const int N = sv.N, A = sv.A, nb1 = 1 << (K - 8);
    auto Dh = [&](int p, int c) -> uint64_t {          // D(p, c), s = 1/2
        const int W = sv.S2 * N + 1;
        if (p < 0 || p > N || c < 0 || c > p) return 0;
        return b->D[(size_t)p * W + c];
    };
    U.assign((size_t)(K + 1) * nb1, 0);
    R0.assign(256, 0);
    C.assign((size_t)(N + 1) * (A + 1), 0);
    // R0[b0]: rank terms of the ones of byte 0 (positions 0..7, counts from 1)
    for (int b0 = 0; b0 < 256; ++b0) {
        uint64_t r = 0;
        int cnt = 0;
        for (int t = 0; t < 8; ++t)
            if (b0 >> t & 1) r += Dh(t, ++cnt);
        R0[b0] = (uint8_t)r;
    }
    // U[k][b1]: rank terms of the ones of byte 1 (positions 8..K-1) when the low word
    // holds k ones, i.e. byte 0 holds k - popc(b1)
    for (int k = 0; k <= K; ++k)
        for (int b1 = 0; b1 < nb1; ++b1) {
            int c = k - __builtin_popcount((unsigned)b1);
            if (c < 0 || c > 8) continue;
            uint64_t r = 0;
            for (int t = 0; t < K - 8; ++t)
                if (b1 >> t & 1) r += Dh(8 + t, ++c);
            if (r > 0xFFFF) return fail(HM_EOVERFLOW, "low rank table entry exceeds 16 bits");
            U[(size_t)k * nb1 + b1] = (uint16_t)r;
        }
    for (int p = 0; p <= N; ++p)
        for (int c = 0; c <= A; ++c) {
            uint64_t v = Dh(p, c);
            C[(size_t)p * (A + 1) + c] = v > 0xFFFFFFFFull ? 0xFFFFFFFFu : (uint32_t)v;
        }
    return HM_OK;
}

static int blk_tables(hm_basis *b, int K, const void **dev, int *bytes, int *oU, int *oR0, int *oC,
                      const uint16_t **lw, int *lwoff) {
    auto it = b->blk_tabs.find(K);
    if (it == b->blk_tabs.end()) {
        std::vector<uint16_t> U;
        std::vector<uint8_t> R0;
        std::vector<uint32_t> C;
        HM_TRY(blk_host_tables(b, K, U, R0, C));
        BlkTab t;
        t.oU = 0;
        t.oR0 = (int)al16(U.size() * 2);
        t.oC = t.oR0 + 256;
        t.bytes = (int)al16(t.oC + C.size() * 4);
        // the K-bit words grouped by popcount, each group in increasing order: the low
        // words of a block in rank order (the rank of Sec. 3.2 orders words of equal
        // popcount numerically)
        std::vector<uint16_t> lw((size_t)1 << K);
        {
            size_t w = 0;
            for (int k = 0; k <= K; ++k) {
                t.lwoff[k] = (int)w;
                for (uint32_t l = 0; l < (1u << K); ++l)
                    if (__builtin_popcount(l) == k) lw[w++] = (uint16_t)l;
            }
            t.lwoff[K + 1] = (int)w;
        }
        const size_t olw = al16(t.bytes);
        const size_t total = olw + lw.size() * 2;
        std::vector<unsigned char> host(total, 0);
        memcpy(host.data() + t.oU, U.data(), U.size() * 2);
        memcpy(host.data() + t.oR0, R0.data(), 256);
        memcpy(host.data() + t.oC, C.data(), C.size() * 4);
        memcpy(host.data() + olw, lw.data(), lw.size() * 2);
        HM_CUDA(cudaMalloc(&t.dev, total));
        cudaError_t e = cudaMemcpy(t.dev, host.data(), total, cudaMemcpyHostToDevice);
        if (e != cudaSuccess) { cudaFree(t.dev); return cuda_fail(e, "block tables"); }
        t.lw = (uint16_t *)((unsigned char *)t.dev + olw);
        it = b->blk_tabs.emplace(K, t).first;
    }
    *dev = it->second.dev;
    *bytes = it->second.bytes;
    *oU = it->second.oU;
    *oR0 = it->second.oR0;
    *oC = it->second.oC;
    *lw = it->second.lw;
    memcpy(lwoff, it->second.lwoff, sizeof it->second.lwoff);
    return HM_OK;
}

// integer coefficient of a per-bond plan: round(h 2^pb_s)
long long pb_coef(const BlkParams &P, double h) { return std::llround(std::ldexp(h, P.pb_s)); }

// Compile-time slots of the thread-per-row kernels (BlkParams::ln ..).  Sets rows_ok = 0
// when a class has more bonds of one kind than the slots hold.
static void blk_plan_slots(const BondParams &bp, const std::vector<int> &bc, int K, BlkParams *P) {
    P->rows_ok = K <= 15 ? 1 : 0;
    P->kshift = K - 6;
    std::map<std::pair<int, int>, uint32_t> cgroups;      // (class, d) -> mask of p
    for (int t = 0; t < bp.nb; ++t) {
        const int c = bc[t], p = bp.p[t], q = bp.q[t];    // p < q
        if (q < K) {
            const int ty = q < 8 ? 0 : (p >= 8 ? 1 : 2);
            int &n = P->ln[c][ty];
            if (n == HM_BLK_SL) { P->rows_ok = 0; continue; }
            const uint32_t pat = (1u << p) | (1u << q);
            P->ld[c][ty][n] = (uint8_t)(q - p);
            if (P->perbond) P->pb_lb[ty][n] = (uint8_t)t;
            P->lvm[c][ty][n] = 1u << p;
            P->lxa[c][ty][n] = (uint16_t)(ty == 0 ? (pat & 255u) << 2 : ty == 2 ? (1u << p) << 2 : 0u);
            P->lxb[c][ty][n] = (uint16_t)(ty == 1 ? (pat >> 8) << 2 : ty == 2 ? (1u << (q - 8)) << 2 : 0u);
            ++n;
            cgroups[{c, q - p}] |= 1u << p;
        } else if (p < K) {
            const int ty = p < 8 ? 0 : 1;
            int &n = P->xn[c][ty];
            if (n == HM_BLK_SX) { P->rows_ok = 0; continue; }
            P->xxa[c][ty][n] = (uint16_t)(ty == 0 ? (1u << p) << 2 : (1u << (p - 8)) << 2);
            if (P->perbond) P->pb_xb[ty][n] = (uint8_t)t;
            P->xf_p[P->nxf] = (uint8_t)p;
            P->xf_q[P->nxf] = (uint8_t)(q - K);
            P->xf_dst[P->nxf] = (uint8_t)((2 * c + ty) * HM_BLK_SX + n);
            ++P->nxf;
            ++n;
        }
    }
    for (auto &kv : cgroups) {
        const int c = kv.first.first;
        if (P->lgn[c] == HM_BLK_SG) { P->rows_ok = 0; continue; }
        P->lgd[c][P->lgn[c]] = (uint8_t)kv.first.second;
        P->lgm[c][P->lgn[c]] = kv.second;
        ++P->lgn[c];
    }
}

static int blk_plan_bonds(hm_basis *b, const BondParams &bp, const std::vector<int> &bc, int K, BlkParams *P);

int blk_plan(hm_basis *b, const BondParams &bp_all, int K, BlkParams *P, bool bond_corr, uint64_t use) {
    const SectorView &sv = b->view;
    const BondParams &bp = bp_all;
    if (sv.S2 != 1 || sv.N > 32 || sv.N < K + 2 || K < 8 || K > 16 || bp.nb > HM_BLK_MAXB ||
        sv.idx64)
        return 1;
    memset(P, 0, sizeof *P);
    P->N = sv.N; P->K = K; P->H = sv.N - K; P->A = sv.A; P->nb1 = 1 << (K - 8);
    P->dim = (uint32_t)sv.dim;
    P->par = b->parity;
    // coupling classes: distinct J values; with more than HM_BLK_MAXC of them every bond
    // keeps its own coefficient (per-bond rows, class 0 slots)
    std::vector<double> cls;
    std::vector<int> bc(bp.nb);
    for (int t = 0; t < bp.nb; ++t) {
        const double J = -bp.jm[t];
        int c = (int)(std::find(cls.begin(), cls.end(), J) - cls.begin());
        if (c == (int)cls.size()) cls.push_back(J);
        bc[t] = c;
    }
    if ((int)cls.size() > HM_BLK_MAXC || bond_corr) {
        P->perbond = 1;
        P->bcmode = bond_corr ? 1 : 0;
        cls.clear();
        std::fill(bc.begin(), bc.end(), 0);
        double g0 = 0.0, mx = 0.0;
        for (int t = 0; t < bp.nb; ++t) {
            g0 += bp.jm[t] / 4.0;                                 // -J_b / 4
            mx = std::max(mx, std::fabs(bp.jm[t] / 2.0));
        }
        P->pb_g0 = g0;
        mx = std::max(mx, std::fabs(g0));
        int ex = 0;
        std::frexp(mx, &ex);                                      // mx < 2^ex
        P->pb_s = mx > 0.0 ? 61 - ex : 0;                         // |C| <= 2^61
        P->pb_c0 = std::llround(std::ldexp(g0, P->pb_s));
    }
    P->nc = (int)cls.size() > 0 ? (int)cls.size() : 1;
    if (P->perbond) P->ntot[0] = 0;
    for (int c = 0; c < (int)cls.size(); ++c) {
        const double g = -cls[c] / 4.0;
        P->g_hi[c] = (float)g;
        P->g_lo[c] = (float)(g - (double)P->g_hi[c]);
        P->gq[c] = (float)g;
    }
    for (int t = 0; t < bp.nb; ++t) P->ntot[bc[t]]++;
    // integer-ratio classes: every -J_c/4 an exact small multiple of the smallest one
    P->iratio = 0;
    if (!cls.empty()) {
        double g0 = 0.0;
        for (double J : cls) {
            const double g = std::fabs(J / 4.0);
            if (g > 0.0 && (g0 == 0.0 || g < g0)) g0 = g;
        }
        bool ok = g0 > 0.0;
        long weight = 0;
        for (int c = 0; c < (int)cls.size() && ok; ++c) {
            const double g = -cls[c] / 4.0;
            const double kr = g / g0;
            const long ki = std::lround(kr);
            if ((double)ki != kr || std::labs(ki) > 64 || (double)ki * g0 != g) ok = false;
            P->Kc[c] = (int)ki;
            weight += std::labs(ki) * P->ntot[c];
        }
        // |T_c| < 3 n_c 2^53 per row: the weighted sum must stay below 2^63
        if (ok && weight * 3 < 1000) {
            P->iratio = 1;
            P->g0 = g0;
            P->g0_hi = (float)g0;
            P->g0_lo = (float)(g0 - (double)P->g0_hi);
            int ex = 0;
            const double fr = std::frexp(g0, &ex);
            P->g0_pow2 = fr == 0.5 ? 1 : 0;
            P->g0_exp = ex - 1;                       // g0 = 2^(ex-1) when a power of two
        }
    }
    // the bonds this plan applies (a subset only on the class path, where the classes and
    // their integer ratios above come from the whole list)
    if (use != ~0ull && (P->perbond || bp.nb > 64)) return 1;
    BondParams sub = bp;
    std::vector<int> sbc;
    sub.nb = 0;
    for (int t = 0; t < bp.nb; ++t) {
        if (t < 64 && !((use >> t) & 1ull)) continue;
        sub.p[sub.nb] = bp.p[t]; sub.q[sub.nb] = bp.q[t];
        sub.jm[sub.nb] = bp.jm[t]; sub.jmf[sub.nb] = bp.jmf[t];
        ++sub.nb;
        sbc.push_back(bc[t]);
    }
    if (use != ~0ull) {
        for (int c = 0; c < HM_BLK_MAXC; ++c) P->ntot[c] = 0;
        for (int t = 0; t < sub.nb; ++t) P->ntot[sbc[t]]++;
    }
    return blk_plan_bonds(b, sub, sbc, K, P);
}

// the slots, groups and tables of a plan whose classes are set: bonds bp with classes bc
static int blk_plan_bonds(hm_basis *b, const BondParams &bp, const std::vector<int> &bc, int K, BlkParams *P) {
    const SectorView &sv = b->view;
    // low groups keyed by (class, type, d); high and cross bonds by class
    std::map<std::tuple<int, int, int>, uint32_t> groups;
    std::vector<std::tuple<int, int, int>> hi[HM_BLK_MAXC], cr[HM_BLK_MAXC];   // (p, q, bond)
    for (int t = 0; t < bp.nb; ++t) {
        const int p = bp.p[t], q = bp.q[t];  // p < q
        if (q < K) {
            const int type = q < 8 ? 0 : (p >= 8 ? 1 : 2);
            groups[std::make_tuple(bc[t], type, q - p)] |= 1u << p;
        } else if (p >= K) {
            hi[bc[t]].push_back({p - K, q - K, t});
        } else {
            cr[bc[t]].push_back({p, q - K, t});
        }
    }
    if ((int)groups.size() > HM_BLK_MAXG) return 1;
    int g = 0;
    for (int c = 0; c < HM_BLK_MAXC; ++c)
        for (int ty = 0; ty < 3; ++ty) {
            P->lg_cs[3 * c + ty] = g;
            for (auto &kv : groups)
                if (std::get<0>(kv.first) == c && std::get<1>(kv.first) == ty) {
                    P->lg_mask[g] = kv.second;
                    P->lg_d[g] = (uint8_t)std::get<2>(kv.first);
                    ++g;
                }
        }
    P->lg_cs[3 * HM_BLK_MAXC] = g;
    P->nlg = g;
    int nh = 0, ncr = 0;
    for (int c = 0; c < HM_BLK_MAXC; ++c) {
        P->hb_start[c] = nh;
        for (auto &e : hi[c]) {
            P->hb_p[nh] = (uint8_t)std::get<0>(e);
            P->hb_q[nh] = (uint8_t)std::get<1>(e);
            if (P->perbond) P->pb_hc[nh] = pb_coef(*P, -bp.jm[std::get<2>(e)] / 2.0);   // J_b / 2
            P->pb_hbb[nh] = (uint8_t)std::get<2>(e);
            ++nh;
        }
        P->cb_start[c] = ncr;
        for (auto &e : cr[c]) { P->cb_p[ncr] = (uint8_t)std::get<0>(e); P->cb_q[ncr] = (uint8_t)std::get<1>(e); ++ncr; }
    }
    P->hb_start[HM_BLK_MAXC] = nh;
    P->cb_start[HM_BLK_MAXC] = ncr;
    P->nhb = nh;
    P->ncb = ncr;
    // largest block: max over the low popcounts that occur of C(K, k)
    int mb = 0;
    for (int k = std::max(0, sv.A - (sv.N - K)); k <= std::min(K, sv.A); ++k) {
        uint64_t c = 1;
        for (int i = 0; i < k; ++i) c = c * (K - i) / (i + 1);
        mb = std::max(mb, (int)c);
    }
    P->max_block = mb;
    const void *dev;
    int bytes, oU, oR0, oC;
    HM_TRY(blk_tables(b, K, &dev, &bytes, &oU, &oR0, &oC, &P->lw, P->lwoff));
    P->tab = dev; P->tab_bytes = bytes; P->off_U = oU; P->off_R0 = oR0; P->off_C = oC;
    blk_plan_slots(bp, bc, K, P);
    return 0;
}

// ---------------------------------------------------------------------------------------
// kernels with the generic row policy (blk_sweep.cuh); jit.cu builds the same bodies
// with the plan's bonds written out
// ---------------------------------------------------------------------------------------
template <class T, int NC>
__global__ void __launch_bounds__(BLK_NT, 3)
k_blk_matvec(BlkParams P, const T *__restrict__ x, T *__restrict__ y, const int *__restrict__ Eptr) {
    matvec_body<T, NC, RowGeneric<NC>>(P, x, y, Eptr);
}

template <int NC, bool IR>
__global__ void __launch_bounds__(BLK_NT, 3)
k_blk_lz64(BlkParams P, const long long *__restrict__ Xc, unsigned long long *__restrict__ Y, LzScalars *S, int pc,
           double *__restrict__ part) {
    lz64_body<NC, IR, RowGeneric<NC>>(P, Xc, Y, S, pc, part);
}

template <int NC>
__global__ void __launch_bounds__(BLK_NT, 3)
k_blk_lz32(BlkParams P, const float *__restrict__ qc, float *__restrict__ qp, LzScalars *S, double *__restrict__ part) {
    lz32_body<NC, RowGeneric<NC>>(P, qc, qp, S, part);
}

// largest exponent field of a double vector (for the fixed-point unit)
__global__ void k_max_exp(const unsigned long long *__restrict__ x, uint64_t n, int *out) {
    int m = 0;
    for (uint64_t i = blockIdx.x * (uint64_t)blockDim.x + threadIdx.x; i < n; i += (uint64_t)gridDim.x * blockDim.x)
        m = max(m, (int)((x[i] >> 52) & 0x7FF));
    for (int o = 16; o > 0; o >>= 1) m = max(m, __shfl_down_sync(0xffffffffu, m, o));
    if ((threadIdx.x & 31) == 0) atomicMax(out, m);
}

template <class T, int NC>
static int launch_blk_matvec(hm_basis *b, const BlkParams &P, const T *x, T *y, cudaStream_t st) {
    const size_t sm = blk_row_smem_bytes(P, sizeof(T) == 8 ? 8 : 4, BLK_XPAD);
    HM_CUDA(raise_smem_limit(k_blk_matvec<T, NC>, sm));
    int *Ed = nullptr;
    if constexpr (sizeof(T) == 8) {
        Ed = (int *)b->d_scratch;
        HM_CUDA(cudaMemsetAsync(Ed, 0, sizeof(int), st));
        k_max_exp<<<grid_blocks(P.dim, 256), 256, 0, st>>>((const unsigned long long *)x, P.dim, Ed);
        HM_CUDA(cudaGetLastError());
    }
    int per = 1;
    HM_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per, k_blk_matvec<T, NC>, BLK_NT, sm));
    const int blocks = std::min<int>(sm_count() * std::max(per, 1), 1 << P.H);
    k_blk_matvec<T, NC><<<blocks, BLK_NT, sm, st>>>(P, x, y, Ed);
    HM_CUDA(cudaGetLastError());
    return HM_OK;
}

// split position: 15 low sites (blocks <= 6435 rows: three 512-thread CTAs per SM), or
// the largest K <= 15 that leaves two high sites
// split position of the block path: the low part holds K = min(15, N - 2) sites
// (HM_BLK_K = 8..15 overrides, for tuning); the thread-per-row slots need K <= 15.  The
// Lanczos workspace sizes its per-block partials (2^(N-K) blocks) with the same function.
int blk_K(const hm_basis *b) {
    int K = 15;
    if (const char *e = getenv("HM_BLK_K")) K = std::max(8, std::min(15, atoi(e)));
    return std::min(K, b->view.N - 2);
}

// f(kernel) for the FP64 block-product instance of the plan (class count, integer ratios)
template <class F>
static int lz64_dispatch(const BlkParams &P, F &&f) {
    if (P.iratio) {
        if (P.nc == 1) return f(k_blk_lz64<1, true>);
        if (P.nc == 2) return f(k_blk_lz64<2, true>);
        return f(k_blk_lz64<4, true>);
    }
    if (P.nc == 1) return f(k_blk_lz64<1, false>);
    if (P.nc == 2) return f(k_blk_lz64<2, false>);
    return f(k_blk_lz64<4, false>);
}

template <class K_t>
static int set_smem(K_t kern, size_t sm) {
    HM_CUDA(raise_smem_limit(kern, (int)sm));
    return HM_OK;
}

// Lanczos hooks: plan (0 = block path usable), attribute setup, launch
int blk_lz_plan(hm_basis *b, const BondParams &bp, int dtype, BlkParams *P, int *blocks) {
    int rc = blk_plan(b, bp, blk_K(b), P);
    if (rc != 0) return rc;
    const size_t sm = blk_row_smem_bytes(*P, dtype == HM_F64 ? 8 : 4, BLK_XPAD);
    if (!P->rows_ok || sm > 200 * 1024) return 1;
    int per = 1;
    if (dtype == HM_F64) {
        HM_TRY(lz64_dispatch(*P, [&](auto kern) -> int {
            HM_TRY(set_smem(kern, sm));
            HM_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per, kern, BLK_NT, sm));
            return HM_OK;
        }));
    } else {
        if (P->nc == 1) { HM_TRY(set_smem(k_blk_lz32<1>, sm)); HM_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per, k_blk_lz32<1>, BLK_NT, sm)); }
        else if (P->nc == 2) { HM_TRY(set_smem(k_blk_lz32<2>, sm)); HM_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per, k_blk_lz32<2>, BLK_NT, sm)); }
        else { HM_TRY(set_smem(k_blk_lz32<4>, sm)); HM_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per, k_blk_lz32<4>, BLK_NT, sm)); }
    }
    *blocks = std::min<int>(sm_count() * std::max(per, 1), 1 << P->H);
    return 0;
}

// kernel specialised to the plan (jit.cu), with its launch attributes; 1 = not available
int jit_lz_kernel(const BlkParams &P, int dtype, const BondParams &bp, const void **kern, int split = 0);
int jit_mv_kernel(const BlkParams &P, int dtype, const BondParams &bp, const void **kern);
// pad elements after the staged rows of a specialised kernel (jit.cu)
int jit_pad(const void *kern);

int blk_lz_jit(const BlkParams &P, int dtype, const BondParams &bp, const void **kern, int *blocks, int split) {
    *kern = nullptr;
    const void *k = nullptr;
    if (jit_lz_kernel(P, dtype, bp, &k, split) != 0) return 1;
    const size_t sm = blk_row_smem_bytes(P, dtype == HM_F64 ? 8 : 4, jit_pad(k));
    if (raise_smem_limit(k, (int)sm) != cudaSuccess) {
        cudaGetLastError();
        return 1;
    }
    int per = 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per, k, BLK_NT, sm) != cudaSuccess || per < 1) {
        cudaGetLastError();
        return 1;
    }
    *blocks = std::min<int>(sm_count() * per, 1 << P.H);
    *kern = k;
    return 0;
}

// Per-class target tables of a plan (the "table" row policy of the specialised kernels,
// jit.cu).  The low part of every block of class k runs through the same C(K, k) low words
// in the same order, so the rank of each low-site exchange target (Sec. 3.2) depends only on
// (k, r) and the bond, not on the block.  The kernels therefore read the targets of a row
// from a table instead of forming them from rank-table reads in shared memory.
//
// The low slots are grouped first into edge-disjoint triangles: bonds (a, b), (b, c), (a, c)
// among the low sites with (a, b) and (b, c) of one class.  Of the three spin pairs of a
// triangle either none or exactly two are unequal, so two gathers serve its three slots: the
// table holds the first and the second allowed target (in the order (a, b), (b, c), (a, c)).
// The first allowed edge is always of the class of (a, b); the second is (b, c) exactly when
// the spins of a and c are parallel, which the kernel reads off the row's own word.  The
// remaining slots take one entry each.  Entries: the triangles' two targets, the single
// slots' targets, the rank of l ^ 2^p for each low end p of a cross bond.  Targets are byte
// offsets into the staged block (rows times esize), the zero row after the block when not
// allowed.  16-bit entries, eight to a 16-byte chunk, chunk-major so that consecutive rows
// read consecutive chunks (2^K rows x chunks x 16 bytes: 1.5 MB at K = 15 for the J1-J2
// ring), built once per basis, layout and element size.  A per-bond plan (each bond its own
// coefficient) takes no triangles, and a slot whose exchange is not allowed points at the
// row itself, so that its difference x_i - x_t vanishes.  Returns 0 and sets P->tt, or 1 when
// the policy does not apply (more than 48 entries, or HM_JIT_ROW selects another policy).
int blk_target_table(hm_basis *b, BlkParams *P, int esize) {
    P->tt = nullptr;
    const char *rowk = getenv("HM_JIT_ROW");
    if (rowk && *rowk && strcmp(rowk, "table") != 0) return 1;
    if (!P->rows_ok || P->bcmode || P->K > 15) return 1;
    const int K = P->K;
    // per-bond plans: every slot keeps its own coefficient, so no triangles; an exchange that
    // is not allowed points at the row itself, whose difference x_i - x_t is then zero
    const bool self = P->perbond != 0;
    struct Slot { int p, q, c; bool used; };
    std::vector<Slot> low;
    for (int c = 0; c < P->nc; ++c)
        for (int ty = 0; ty < 3; ++ty)
            for (int k = 0; k < P->ln[c][ty]; ++k) {
                const int p = __builtin_ctz(P->lvm[c][ty][k]);
                low.push_back({p, p + P->ld[c][ty][k], c, false});
            }
    auto find = [&](int x, int y) {
        for (size_t i = 0; i < low.size(); ++i)
            if (!low[i].used && low[i].p == std::min(x, y) && low[i].q == std::max(x, y)) return (int)i;
        return -1;
    };
    // triangles, greedily by their smallest site; e[0] = (a, b), e[1] = (b, c) share site b and
    // a class, e[2] = (a, c) is the opposite edge
    struct Tri { int e[3]; };
    std::vector<Tri> tris;
    for (int x = 0; x < K && !self; ++x)
        for (int y = x + 1; y < K; ++y)
            for (int z = y + 1; z < K; ++z) {
                const int sites[3] = {x, y, z};
                for (int m = 0; m < 3 && tris.size() < 16; ++m) {       // m: the shared site b
                    const int bb = sites[m], aa = sites[(m + 1) % 3], cc = sites[(m + 2) % 3];
                    const int i0 = find(aa, bb), i1 = find(bb, cc), i2 = find(aa, cc);
                    if (i0 < 0 || i1 < 0 || i2 < 0 || low[i0].c != low[i1].c) continue;
                    low[i0].used = low[i1].used = low[i2].used = true;
                    tris.push_back({{i0, i1, i2}});
                    break;
                }
            }
    std::vector<int> sgl;
    for (size_t i = 0; i < low.size(); ++i)
        if (!low[i].used) sgl.push_back((int)i);
    std::vector<int> cps;
    for (int e = 0; e < P->nxf; ++e)
        if (std::find(cps.begin(), cps.end(), (int)P->xf_p[e]) == cps.end()) cps.push_back(P->xf_p[e]);
    if (cps.size() > 8 || sgl.size() > 48) return 1;
    const int ntri = (int)tris.size(), nsgl = (int)sgl.size();
    const int n = 2 * ntri + nsgl + (int)cps.size();
    if (n > 48) return 1;
    const int nch = (n + 7) / 8;
    const uint32_t zrow = (uint32_t)(P->max_block + BLK_XPAD - 1);
    if ((zrow + 1) * (uint32_t)esize > 65535u) return 1;
    std::string key = std::string(self ? "self:" : "tri:") + std::to_string(K) + ":" + std::to_string(esize) + ":" +
                      std::to_string(P->nc) + ":";
    for (auto &sl : low) key += std::to_string(sl.p) + "-" + std::to_string(sl.q) + "/" + std::to_string(sl.c) + ",";
    key += "|";
    for (int p : cps) key += std::to_string(p) + ",";
    auto it = b->blk_ttabs.find(key);
    if (it == b->blk_ttabs.end()) {
        const uint32_t rows = 1u << K;
        std::vector<uint32_t> rank(rows);                 // colex rank within the popcount class
        {
            std::vector<uint32_t> seen(K + 1, 0);
            for (uint32_t l = 0; l < rows; ++l) rank[l] = seen[__builtin_popcount(l)]++;
        }
        std::vector<uint16_t> host((size_t)nch * rows * 8, 0);
        for (uint32_t l = 0; l < rows; ++l) {
            const uint32_t g = rank[l] + (uint32_t)P->lwoff[__builtin_popcount(l)];   // position in the word list
            auto put = [&](int s, uint32_t v) { host[((size_t)(s / 8) * rows + g) * 8 + (s % 8)] = (uint16_t)v; };
            auto ok = [&](const Slot &sl) { return ((l >> sl.p) ^ (l >> sl.q)) & 1u; };
            auto tgt = [&](const Slot &sl) { return rank[l ^ ((1u << sl.p) | (1u << sl.q))] * (uint32_t)esize; };
            const uint32_t z = zrow * (uint32_t)esize;
            for (int t = 0; t < ntri; ++t) {
                const Slot &e0 = low[tris[t].e[0]], &e1 = low[tris[t].e[1]], &e2 = low[tris[t].e[2]];
                const bool v0 = ok(e0), v1 = ok(e1), v2 = ok(e2);
                uint32_t o1 = z, o2 = z;
                if (v0 && v1) { o1 = tgt(e0); o2 = tgt(e1); }
                else if (v0 && v2) { o1 = tgt(e0); o2 = tgt(e2); }
                else if (v1 && v2) { o1 = tgt(e1); o2 = tgt(e2); }
                put(2 * t, o1);
                put(2 * t + 1, o2);
            }
            const uint32_t own = rank[l] * (uint32_t)esize;
            for (int i = 0; i < nsgl; ++i) put(2 * ntri + i, ok(low[sgl[i]]) ? tgt(low[sgl[i]]) : self ? own : z);
            for (size_t i = 0; i < cps.size(); ++i)
                put(2 * ntri + nsgl + (int)i, rank[l ^ (1u << cps[i])] * (uint32_t)esize);
        }
        void *dev = nullptr;
        HM_CUDA(cudaMalloc(&dev, host.size() * 2));
        cudaError_t e = cudaMemcpy(dev, host.data(), host.size() * 2, cudaMemcpyHostToDevice);
        if (e != cudaSuccess) { cudaFree(dev); return cuda_fail(e, "target table"); }
        it = b->blk_ttabs.emplace(key, dev).first;
    }
    P->tt = (const uint4 *)it->second;
    P->tt_stride = 1u << K;
    P->tt_n = n;
    P->tt_ncross = (int)cps.size();
    for (size_t i = 0; i < cps.size(); ++i) P->tt_cross_p[i] = cps[i];
    P->tt_ntri = ntri;
    P->tt_nsgl = nsgl;
    for (int t = 0; t < ntri; ++t) {
        P->tt_tri_ca[t] = (uint8_t)low[tris[t].e[0]].c;
        P->tt_tri_cb[t] = (uint8_t)low[tris[t].e[2]].c;
        P->tt_tri_a[t] = (uint8_t)low[tris[t].e[2]].p;
        P->tt_tri_c[t] = (uint8_t)low[tris[t].e[2]].q;
    }
    for (int i = 0; i < nsgl; ++i) P->tt_sgl_c[i] = (uint8_t)low[sgl[i]].c;
    return 0;
}

// Split FP64 product for large s = 1/2 sectors with integer-ratio couplings.  In one pass
// the exchanges that reach the top high sites gather blocks far away in the row order, which
// have left L2 by then (about 105 bytes of DRAM traffic per row at N = 32 against 16).  The
// bonds with an end at site N - 7 or above therefore go to a second pass, which takes the
// blocks with the top high sites varying fastest (rot = 9), so that those targets are
// neighbours in time; the first pass keeps the row order for the rest.  Pass 1 leaves the
// exact integer row sums of its bonds in Y, pass 2 adds its own and rounds once: the result
// is the single pass's, bit for bit.  Measured at N = 32 the split cuts DRAM traffic but
// takes longer (20.0 against 18.6 ms per product): the one-pass kernel is bound by its
// shared-memory wavefronts and issue, not by DRAM, and the second pass repeats the per-block
// work.  So it is off unless HM_BLK_SPLIT = 1 asks for it (2 applies it only to sectors of
// 2^27 rows and more).  Returns 0 with both plans and their specialised kernels, 1 when the
// split does not apply.
int blk_lz_split(hm_basis *b, const BondParams &bp, const BlkParams &P, int dtype, BlkParams *PA, BlkParams *PB,
                 const void **kA, const void **kB, int *blkA, int *blkB) {
    const char *e = getenv("HM_BLK_SPLIT");
    const int mode = e && *e ? atoi(e) : 0;
    if ((mode != 1 && mode != 2) || dtype != HM_F64) return 1;
    if (mode == 2 && P.dim < (1u << 27)) return 1;
    if (!P.iratio || !P.g0_pow2 || P.perbond || P.par || bp.nb > 64 || !P.rows_ok) return 1;
    const int S = P.N - 7;
    const uint64_t all = bp.nb == 64 ? ~0ull : ((1ull << bp.nb) - 1ull);
    uint64_t far = 0;
    for (int t = 0; t < bp.nb; ++t)
        if (std::max(bp.p[t], bp.q[t]) >= S) far |= 1ull << t;
    if (far == 0 || far == all) return 1;
    if (blk_plan(b, bp, P.K, PA, false, all & ~far) != 0 || blk_plan(b, bp, P.K, PB, false, far) != 0) return 1;
    if (!PA->rows_ok || !PB->rows_ok || !PA->iratio || !PB->iratio) return 1;
    PA->split = 1;
    PB->split = 2;
    PB->rot = std::min(PB->H, 9);
    if (blk_target_table(b, PA, 8) < 0 || blk_target_table(b, PB, 8) < 0) return 1;
    if (blk_lz_jit(*PA, dtype, bp, kA, blkA, 1) != 0 || blk_lz_jit(*PB, dtype, bp, kB, blkB, 2) != 0) return 1;
    return 0;
}

// jit: the specialised kernel, or nullptr for the generic one
int blk_lz64_launch(const BlkParams &P, const long long *Xc, unsigned long long *Y, LzScalars *S, int pc,
                    double *part, int blocks, cudaStream_t st, const void *jit) {
    const size_t sm = blk_row_smem_bytes(P, 8, jit_pad(jit));
    if (jit) {
        void *args[] = {(void *)&P, (void *)&Xc, (void *)&Y, (void *)&S, (void *)&pc, (void *)&part};
        HM_CUDA(cudaLaunchKernel(jit, dim3(blocks), dim3(BLK_NT), args, sm, st));
        return HM_OK;
    }
    HM_TRY(lz64_dispatch(P, [&](auto kern) -> int {
        kern<<<blocks, BLK_NT, sm, st>>>(P, Xc, Y, S, pc, part);
        return HM_OK;
    }));
    HM_CUDA(cudaGetLastError());
    return HM_OK;
}

int blk_lz32_launch(const BlkParams &P, const float *qc, float *qp, LzScalars *S, double *part, int blocks,
                    cudaStream_t st, const void *jit) {
    const size_t sm = blk_row_smem_bytes(P, 4, jit_pad(jit));
    if (jit) {
        void *args[] = {(void *)&P, (void *)&qc, (void *)&qp, (void *)&S, (void *)&part};
        HM_CUDA(cudaLaunchKernel(jit, dim3(blocks), dim3(BLK_NT), args, sm, st));
        return HM_OK;
    }
    if (P.nc == 1) k_blk_lz32<1><<<blocks, BLK_NT, sm, st>>>(P, qc, qp, S, part);
    else if (P.nc == 2) k_blk_lz32<2><<<blocks, BLK_NT, sm, st>>>(P, qc, qp, S, part);
    else k_blk_lz32<4><<<blocks, BLK_NT, sm, st>>>(P, qc, qp, S, part);
    HM_CUDA(cudaGetLastError());
    return HM_OK;
}

// per-bond plan: the specialised y = H x kernel (jit.cu); 1 when it is not available
static int launch_blk_matvec_pb(hm_basis *b, const BlkParams &P0, const BondParams &bp, const void *x, void *y,
                                int dtype, cudaStream_t st) {
    BlkParams P = P0;
    const int trc = blk_target_table(b, &P, dtype == HM_F64 ? 8 : 4);
    if (trc < 0) return trc;
    const void *k = nullptr;
    if (jit_mv_kernel(P, dtype, bp, &k) != 0) return 1;
    const size_t sm = blk_row_smem_bytes(P, dtype == HM_F64 ? 8 : 4, BLK_XPAD);
    HM_CUDA(raise_smem_limit(k, (int)sm));
    int *Ed = nullptr;
    if (dtype == HM_F64) {
        Ed = (int *)b->d_scratch;
        HM_CUDA(cudaMemsetAsync(Ed, 0, sizeof(int), st));
        k_max_exp<<<grid_blocks(P.dim, 256), 256, 0, st>>>((const unsigned long long *)x, P.dim, Ed);
        HM_CUDA(cudaGetLastError());
    }
    int per = 0;
    HM_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per, k, BLK_NT, sm));
    const int blocks = std::min<int>(sm_count() * std::max(per, 1), 1 << P.H);
    void *args[] = {(void *)&P, (void *)&x, (void *)&y, (void *)&Ed};
    HM_CUDA(cudaLaunchKernel(k, dim3(blocks), dim3(BLK_NT), args, sm, st));
    return HM_OK;
}

// ---- bond correlations on the block path -------------------------------------------------
int jit_bc_kernel(const BlkParams &P, int dtype, int nbk, const void **kern);

constexpr int BC_CHUNK = 16;               // bonds per bond-correlation launch
constexpr uint64_t BC_MIN_ROWS = 100000;   // smaller sectors: the general kernel (no compile)

// out[k] = sign 2^u (T0 / 4 - C_k / 2) / div from the CTA partials of one chunk (fixed order)
__global__ void k_bc_final(const double *__restrict__ part, int nctas, int nbk, const int *Eptr, double sign,
                           const double *div, double *__restrict__ out) {
    __shared__ double t0s;
    if (threadIdx.x == 0) {
        double t = 0.0;
        for (int c = 0; c < nctas; ++c) t += part[(size_t)c * (nbk + 1) + nbk];
        t0s = t;
    }
    __syncthreads();
    const int k = threadIdx.x;
    if (k >= nbk) return;
    double ck = 0.0;
    for (int c = 0; c < nctas; ++c) ck += part[(size_t)c * (nbk + 1) + k];
    double v = 0.25 * t0s - 0.5 * ck;
    if (Eptr) v = ldexp(v, *Eptr - 1022 - ef::FIX_BITS);
    out[k] = sign * (div ? v / *div : v);
}

// bytes of partial sums the block-path bond correlations need at most
size_t blk_bond_corr_bytes() { return (size_t)sm_count() * 4 * (BC_CHUNK + 1) * sizeof(double); }

// out[b] = sign g^T (s_u.s_v) x / div for every bond, s = 1/2 sectors through the block
// kernels compiled per chunk of bonds; 1 = not applicable (the caller runs the general kernel)
int blk_bond_corr(hm_basis *b, const BondParams &bp, const void *g, const void *x, double *out, int dtype,
                  void *work, size_t work_bytes, double sign, const double *div, cudaStream_t st) {
    const SectorView &sv = b->view;
    if (sv.S2 != 1 || b->parity || bp.nb == 0 || sv.dim < BC_MIN_ROWS) return 1;
    const int nch = (bp.nb + BC_CHUNK - 1) / BC_CHUNK;
    std::vector<BlkParams> plans(nch);
    std::vector<const void *> kerns(nch);
    std::vector<int> blocks(nch);
    const int es = dtype == HM_F64 ? 8 : 4;
    for (int c = 0; c < nch; ++c) {               // every chunk planned and compiled before any launch
        BondParams bc = bp;
        const int c0 = c * BC_CHUNK, nbk = std::min(BC_CHUNK, bp.nb - c0);
        bc.nb = nbk;
        for (int i = 0; i < nbk; ++i) {
            bc.p[i] = bp.p[c0 + i]; bc.q[i] = bp.q[c0 + i];
            bc.jm[i] = bp.jm[c0 + i]; bc.jmf[i] = bp.jmf[c0 + i];
        }
        BlkParams &P = plans[c];
        if (blk_plan(b, bc, blk_K(b), &P, true) != 0 || !P.rows_ok) return 1;
        const size_t sm = blk_row_smem_bytes(P, es, BLK_XPAD);
        if (sm > 200 * 1024 || jit_bc_kernel(P, dtype, nbk, &kerns[c]) != 0) return 1;
        if (raise_smem_limit(kerns[c], (int)sm) != cudaSuccess) {
            cudaGetLastError();
            return 1;
        }
        int per = 0;
        if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per, kerns[c], BLK_NT, sm) != cudaSuccess || per < 1) {
            cudaGetLastError();
            return 1;
        }
        blocks[c] = std::min<int>(sm_count() * std::min(per, 4), 1 << P.H);
        if (!work || work_bytes < (size_t)blocks[c] * (nbk + 1) * sizeof(double)) return 1;
    }
    int *Ed = nullptr;
    if (dtype == HM_F64) {
        Ed = (int *)b->d_scratch;
        HM_CUDA(cudaMemsetAsync(Ed, 0, sizeof(int), st));
        k_max_exp<<<grid_blocks(sv.dim, 256), 256, 0, st>>>((const unsigned long long *)x, sv.dim, Ed);
        HM_CUDA(cudaGetLastError());
    }
    double *part = (double *)work;
    for (int c = 0; c < nch; ++c) {
        const int nbk = std::min(BC_CHUNK, bp.nb - c * BC_CHUNK);
        const size_t sm = blk_row_smem_bytes(plans[c], es, BLK_XPAD);
        void *args[] = {(void *)&plans[c], (void *)&x, (void *)&g, (void *)&Ed, (void *)&part};
        HM_CUDA(cudaLaunchKernel(kerns[c], dim3(blocks[c]), dim3(BLK_NT), args, sm, st));
        k_bc_final<<<1, 32, 0, st>>>(part, blocks[c], nbk, Ed, sign, div, out + c * BC_CHUNK);
        HM_CUDA(cudaGetLastError());
    }
    return HM_OK;
}

// name of the kernel blk_matvec launches for these arguments, or nullptr when the block
// path does not apply
const char *blk_matvec_kernel(hm_basis *b, const BondParams &bp, int dtype, int nvec) {
    if (nvec != 1) return nullptr;
    BlkParams P;
    if (blk_plan(b, bp, blk_K(b), &P) != 0) return nullptr;
    if (!P.rows_ok || blk_row_smem_bytes(P, dtype == HM_F64 ? 8 : 4, BLK_XPAD) > 200 * 1024) return nullptr;
    if (!P.perbond) return "k_blk_matvec";
    const void *k = nullptr;
    return jit_mv_kernel(P, dtype, bp, &k) == 0 ? "k_blk_matvec_jit" : nullptr;
}

// returns 1 when the block path does not apply (caller falls back to the row kernel)
int blk_matvec(hm_basis *b, const BondParams &bp, const void *x, void *y, int dtype, int nvec,
               cudaStream_t st) {
    if (nvec != 1) return 1;
    BlkParams P;
    int rc = blk_plan(b, bp, blk_K(b), &P);
    if (rc != 0) return rc;
    if (!P.rows_ok || blk_row_smem_bytes(P, dtype == HM_F64 ? 8 : 4, BLK_XPAD) > 200 * 1024) return 1;
    if (P.perbond) return launch_blk_matvec_pb(b, P, bp, x, y, dtype, st);
    if (dtype == HM_F64) {
        switch (P.nc) {
            case 1: return launch_blk_matvec<double, 1>(b, P, (const double *)x, (double *)y, st);
            case 2: return launch_blk_matvec<double, 2>(b, P, (const double *)x, (double *)y, st);
            default: return launch_blk_matvec<double, 4>(b, P, (const double *)x, (double *)y, st);
        }
    }
    switch (P.nc) {
        case 1: return launch_blk_matvec<float, 1>(b, P, (const float *)x, (float *)y, st);
        case 2: return launch_blk_matvec<float, 2>(b, P, (const float *)x, (float *)y, st);
        default: return launch_blk_matvec<float, 4>(b, P, (const float *)x, (float *)y, st);
    }
}

}  // namespace hm
