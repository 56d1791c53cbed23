// blk.cu -- host planning and the matvec kernel of the s = 1/2 block path (blk.cuh).
#include <algorithm>
#include <climits>
#include <cstring>
#include <cmath>
#include <map>
#include <tuple>
#include <type_traits>

#include "blk.cuh"

namespace hm {

constexpr int BLK_NT = 512;

__host__ __device__ __forceinline__ size_t al16(size_t x) { return (x + 15) & ~(size_t)15; }

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

static int blk_tables(hm_basis *b, int K, const void **dev, int *bytes, int *oU, int *oR0, int *oC) {
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
        std::vector<unsigned char> host(t.bytes, 0);
        memcpy(host.data() + t.oU, U.data(), U.size() * 2);
        memcpy(host.data() + t.oR0, R0.data(), 256);
        memcpy(host.data() + t.oC, C.data(), C.size() * 4);
        HM_CUDA(cudaMalloc(&t.dev, t.bytes));
        cudaError_t e = cudaMemcpy(t.dev, host.data(), t.bytes, cudaMemcpyHostToDevice);
        if (e != cudaSuccess) { cudaFree(t.dev); return cuda_fail(e, "block tables"); }
        it = b->blk_tabs.emplace(K, t).first;
    }
    *dev = it->second.dev;
    *bytes = it->second.bytes;
    *oU = it->second.oU;
    *oR0 = it->second.oR0;
    *oC = it->second.oC;
    return HM_OK;
}

int blk_plan(hm_basis *b, const BondParams &bp, int K, BlkParams *P) {
    const SectorView &sv = b->view;
    if (sv.S2 != 1 || sv.N > 32 || sv.N < K + 2 || K < 8 || K > 16 || bp.nb > HM_BLK_MAXB ||
        sv.idx64)
        return 1;
    memset(P, 0, sizeof *P);
    P->N = sv.N; P->K = K; P->H = sv.N - K; P->A = sv.A; P->nb1 = 1 << (K - 8);
    P->dim = (uint32_t)sv.dim;
    // coupling classes: distinct J values
    std::vector<double> cls;
    std::vector<int> bc(bp.nb);
    for (int t = 0; t < bp.nb; ++t) {
        const double J = -bp.jm[t];
        int c = (int)(std::find(cls.begin(), cls.end(), J) - cls.begin());
        if (c == (int)cls.size()) {
            if ((int)cls.size() == HM_BLK_MAXC) return 1;
            cls.push_back(J);
        }
        bc[t] = c;
    }
    P->nc = (int)cls.size() > 0 ? (int)cls.size() : 1;
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
    // low groups keyed by (class, type, d); high and cross bonds by class
    std::map<std::tuple<int, int, int>, uint32_t> groups;
    std::vector<std::pair<int, int>> hi[HM_BLK_MAXC], cr[HM_BLK_MAXC];
    for (int t = 0; t < bp.nb; ++t) {
        const int p = bp.p[t], q = bp.q[t];  // p < q
        if (q < K) {
            const int type = q < 8 ? 0 : (p >= 8 ? 1 : 2);
            groups[std::make_tuple(bc[t], type, q - p)] |= 1u << p;
        } else if (p >= K) {
            hi[bc[t]].push_back({p - K, q - K});
        } else {
            cr[bc[t]].push_back({p, q - K});
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
        for (auto &e : hi[c]) { P->hb_p[nh] = (uint8_t)e.first; P->hb_q[nh] = (uint8_t)e.second; ++nh; }
        P->cb_start[c] = ncr;
        for (auto &e : cr[c]) { P->cb_p[ncr] = (uint8_t)e.first; P->cb_q[ncr] = (uint8_t)e.second; ++ncr; }
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
    HM_TRY(blk_tables(b, K, &dev, &bytes, &oU, &oR0, &oC));
    P->tab = dev; P->tab_bytes = bytes; P->off_U = oU; P->off_R0 = oR0; P->off_C = oC;
    return 0;
}

// shared memory: tables | staged rows | BlkShared
size_t blk_smem_bytes(const BlkParams &P, int stage_bytes_per_row, int nvec) {
    return al16(P.tab_bytes) + al16((size_t)P.max_block * stage_bytes_per_row * nvec) +
           blk_shared_bytes(P.max_block);
}

// ---------------------------------------------------------------------------------------
// gathers: how a row value is read from global memory
// ---------------------------------------------------------------------------------------
struct GatherF64 {          // binary64 -> fixed point on the fly (vector exponent E)
    const unsigned long long *x;
    int E;
    __device__ __forceinline__ int64_t operator()(uint32_t j) const { return ef::fix_from_bits(__ldg(x + j), E); }
};
struct GatherFix {          // precomputed fixed-point copy
    const long long *x;
    __device__ __forceinline__ int64_t operator()(uint32_t j) const { return (int64_t)__ldg(x + j); }
};
struct GatherF32 {
    const float *x;
    __device__ __forceinline__ float operator()(uint32_t j) const { return __ldg(x + j); }
};

// hop sums of one row: acc[c] = sum of x over the allowed exchanges of class c, cnt[c]
// their number
template <class Sv, int NC, class G>
__device__ __forceinline__ void blk_row(const BlkParams &P, const BlkTabs &tb, int k, uint32_t off, int r,
                                        uint32_t l, const Sv *Xs, const BlkShared &sh, const G &gx, Sv *acc,
                                        int *cnt) {
    const uint16_t *Uk = tb.U + k * P.nb1;
    const uint32_t i = off + (uint32_t)r;
#pragma unroll
    for (int c = 0; c < NC; ++c) {
        Sv a = Sv(0);
        int mc = blk_low_hops(P, tb, c, l, (uint32_t)r, Uk, [&](uint32_t r2) { a += Xs[r2]; });
        mc += blk_cross_hops(P, tb, c, l, sh, [&](uint32_t j) { a += gx(j); });
        // exchanges among the high positions: the same low word in another block
        const int e0 = sh.hcs[c], e1 = sh.hcs[c + 1];
        int e = e0;
        for (; e + 4 <= e1; e += 4) {
            const Sv v0 = gx(i + sh.hcd[e]), v1 = gx(i + sh.hcd[e + 1]);
            const Sv v2 = gx(i + sh.hcd[e + 2]), v3 = gx(i + sh.hcd[e + 3]);
            a += (v0 + v1) + (v2 + v3);
        }
        for (; e < e1; ++e) a += gx(i + sh.hcd[e]);
        acc[c] = a;
        cnt[c] = mc + (e1 - e0);
    }
}

// T_c = 2 acc_c + (ntot_c - 2 cnt_c) x_i: the class sum of Eq. (E-2-1) rows in units of
// -J_c / 4 (s = 1/2: s^z s^z = +-1/4, exchange element 1/2)
template <int NC>
__device__ __forceinline__ void blk_classes(const BlkParams &P, const int64_t *acc, const int *cnt, int64_t Xo,
                                            int64_t *T) {
#pragma unroll
    for (int c = 0; c < NC; ++c) T[c] = 2 * acc[c] + (int64_t)(P.ntot[c] - 2 * cnt[c]) * Xo;
}

// y (binary64 bits) of a row from its class sums; u = unit exponent of the fixed point.
// Integer-ratio classes with a power-of-two g0 round the exact integer once.
template <int NC>
__device__ __forceinline__ unsigned long long blk_y_bits(const BlkParams &P, const int64_t *T, int u, int64_t *Tsum) {
    if (P.iratio) {
        int64_t s = 0;
#pragma unroll
        for (int c = 0; c < NC; ++c) s += (int64_t)P.Kc[c] * T[c];
        *Tsum = s;
        if (P.g0_pow2) return ef::bits_from_int(s, u + P.g0_exp);
        const ef::df t = ef::df_from_fix(s, u + 1022 + ef::FIX_BITS, 0, 0);
        return ef::bits_from_df(ef::df_mul(t, ef::df{P.g0_hi, P.g0_lo}), 0);
    }
    *Tsum = 0;
    ef::df y{0.0f, 0.0f};
#pragma unroll
    for (int c = 0; c < NC; ++c)
        y = ef::df_add(y, ef::df_mul(ef::df_from_fix(T[c], u + 1022 + ef::FIX_BITS, 0, 0), ef::df{P.g_hi[c], P.g_lo[c]}));
    return ef::bits_from_df(y, 0);
}

template <int NC>
__device__ __forceinline__ float blk_y_f32(const BlkParams &P, const float *acc, const int *cnt, float xo) {
    float y = 0.0f;
#pragma unroll
    for (int c = 0; c < NC; ++c) y += P.gq[c] * (2.0f * acc[c] + (float)(P.ntot[c] - 2 * cnt[c]) * xo);
    return y;
}

// largest exponent field of a double vector (for the fixed-point unit)
__global__ void k_max_exp(const unsigned long long *__restrict__ x, uint64_t n, int *out) {
    int m = 0;
    for (uint64_t i = blockIdx.x * (uint64_t)blockDim.x + threadIdx.x; i < n; i += (uint64_t)gridDim.x * blockDim.x)
        m = max(m, (int)((x[i] >> 52) & 0x7FF));
    for (int o = 16; o > 0; o >>= 1) m = max(m, __shfl_down_sync(0xffffffffu, m, o));
    if ((threadIdx.x & 31) == 0) atomicMax(out, m);
}

// ---------------------------------------------------------------------------------------
// y = H x (matvec API)
// ---------------------------------------------------------------------------------------
template <class T, int NC>
__global__ void __launch_bounds__(BLK_NT)
k_blk_matvec(BlkParams P, const T *__restrict__ x, T *__restrict__ y, const int *__restrict__ Eptr) {
    using Sv = typename std::conditional<sizeof(T) == 8, int64_t, float>::type;
    extern __shared__ __align__(16) unsigned char smem[];
    const BlkTabs tb = stage_blk_tables(P, smem);
    Sv *Xs = (Sv *)(smem + al16(P.tab_bytes));
    const BlkShared sh = blk_carve(smem + al16(P.tab_bytes) + al16((size_t)P.max_block * sizeof(Sv)), P.max_block);
    const int E = Eptr ? *Eptr : 0;
    const int u = E - 1022 - ef::FIX_BITS;
    for (uint32_t h = blockIdx.x; h < (1u << P.H); h += gridDim.x) {
        const int k = P.A - __popc(h);
        if (k < 0 || k > P.K) continue;
        __syncthreads();    // previous block done with the shared buffers
        uint32_t off;
        const int n = blk_setup_block(P, tb, h, k, sh, &off);
        if constexpr (sizeof(T) == 8) {
            const GatherF64 gx{(const unsigned long long *)x, E};
            for (int r = threadIdx.x; r < n; r += blockDim.x) Xs[r] = gx(off + r);
            __syncthreads();
            for (int r = threadIdx.x; r < n; r += blockDim.x) {
                int64_t acc[NC], Tc[NC], ts;
                int cnt[NC];
                blk_row<int64_t, NC>(P, tb, k, off, r, sh.list[r], Xs, sh, gx, acc, cnt);
                blk_classes<NC>(P, acc, cnt, Xs[r], Tc);
                ((unsigned long long *)y)[off + r] = blk_y_bits<NC>(P, Tc, u, &ts);
            }
        } else {
            const GatherF32 gx{(const float *)x};
            for (int r = threadIdx.x; r < n; r += blockDim.x) Xs[r] = gx(off + r);
            __syncthreads();
            for (int r = threadIdx.x; r < n; r += blockDim.x) {
                float acc[NC];
                int cnt[NC];
                blk_row<float, NC>(P, tb, k, off, r, sh.list[r], Xs, sh, gx, acc, cnt);
                y[off + r] = blk_y_f32<NC>(P, acc, cnt, Xs[r]);
            }
        }
    }
}

template <class T, int NC>
static int launch_blk_matvec(hm_basis *b, const BlkParams &P, const T *x, T *y, cudaStream_t st) {
    const size_t sm = blk_smem_bytes(P, sizeof(T) == 8 ? 8 : 4, 1);
    HM_CUDA(cudaFuncSetAttribute(k_blk_matvec<T, NC>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm));
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
static int blk_K(const hm_basis *b) { return std::min(15, b->view.N - 2); }

// ---------------------------------------------------------------------------------------
// Lanczos, FP64: y = H q_cur from the fixed-point copy Xc of q_cur (every gather an
// integer load), written as binary64 to Y; the exact integer dots q.y and q.q_prev
// (Xp: fixed-point copy of q_prev) give alpha without re-reading y.
// part[blk] = (q . H q) and part[gridDim + blk] = (q . q_prev), both in true units.
// ---------------------------------------------------------------------------------------
__device__ __forceinline__ double i128_to_double(__int128 v) {
    const long long hi = (long long)(v >> 64);
    const unsigned long long lo = (unsigned long long)v;
    return (double)hi * 18446744073709551616.0 + (double)lo;
}

template <int NC>
__global__ void __launch_bounds__(BLK_NT)
k_blk_lz64(BlkParams P, const long long *__restrict__ Xc, const long long *__restrict__ Xp,
           unsigned long long *__restrict__ Y, LzScalars *S, int pc, double *__restrict__ part) {
    if (S->done) return;
    extern __shared__ __align__(16) unsigned char smem[];
    __shared__ double red[BLK_NT / 32];
    const BlkTabs tb = stage_blk_tables(P, smem);
    int64_t *Xs = (int64_t *)(smem + al16(P.tab_bytes));
    const BlkShared sh = blk_carve(smem + al16(P.tab_bytes) + al16((size_t)P.max_block * 8), P.max_block);
    const int E = S->emax[pc], Ep = S->emax[pc ^ 1];
    const int u = E - 1022 - ef::FIX_BITS, up = Ep - 1022 - ef::FIX_BITS;
    const GatherFix gx{Xc};
    __int128 d1 = 0, d2 = 0;
    ef::df d1f{0.0f, 0.0f};
    for (uint32_t h = blockIdx.x; h < (1u << P.H); h += gridDim.x) {
        const int k = P.A - __popc(h);
        if (k < 0 || k > P.K) continue;
        __syncthreads();
        uint32_t off;
        const int n = blk_setup_block(P, tb, h, k, sh, &off);
        for (int r = threadIdx.x; r < n; r += blockDim.x) Xs[r] = gx(off + r);
        __syncthreads();
        for (int r = threadIdx.x; r < n; r += blockDim.x) {
            int64_t acc[NC], Tc[NC], ts;
            int cnt[NC];
            blk_row<int64_t, NC>(P, tb, k, off, r, sh.list[r], Xs, sh, gx, acc, cnt);
            const int64_t xo = Xs[r];
            blk_classes<NC>(P, acc, cnt, xo, Tc);
            const unsigned long long yb = blk_y_bits<NC>(P, Tc, u, &ts);
            Y[off + r] = yb;
            if (P.iratio) d1 += (__int128)xo * ts;
            else d1f = ef::df_add(d1f, ef::df_mul(ef::df_from_fix(xo, E, 0, E - 1023), ef::df_from_bits(yb, E - 1023)));
            d2 += (__int128)xo * (int64_t)__ldg(Xp + off + r);
        }
    }
    // true units: q.y = g0 2^(2u) sum X Tsum (integer ratios) or the double-float sum
    // scaled back by 2^(2(E-1023)); q.q_prev = 2^(u+up) sum X Xp
    const double q_y = P.iratio ? ldexp(i128_to_double(d1) * P.g0, 2 * u)
                                : ldexp((double)d1f.hi + (double)d1f.lo, 2 * (E - 1023));
    const double q_qp = ldexp(i128_to_double(d2), u + up);
    const double s1 = block_sum<BLK_NT>(q_y, red);
    __syncthreads();
    const double s2 = block_sum<BLK_NT>(q_qp, red);
    if (threadIdx.x == 0) {
        part[blockIdx.x] = s1;
        part[gridDim.x + blockIdx.x] = s2;
    }
}

// ---------------------------------------------------------------------------------------
// Lanczos, FP32: u = sigma H q - gamma q_prev over q_prev, dot in double-float
// ---------------------------------------------------------------------------------------
template <int NC>
__global__ void __launch_bounds__(BLK_NT)
k_blk_lz32(BlkParams P, const float *__restrict__ qc, float *__restrict__ qp, LzScalars *S, double *__restrict__ part) {
    if (S->done) return;
    extern __shared__ __align__(16) unsigned char smem[];
    __shared__ double red[BLK_NT / 32];
    const BlkTabs tb = stage_blk_tables(P, smem);
    float *Xs = (float *)(smem + al16(P.tab_bytes));
    const BlkShared sh = blk_carve(smem + al16(P.tab_bytes) + al16((size_t)P.max_block * 4), P.max_block);
    const float sig = (float)S->sigma_cur, gam = (float)(S->beta_prev * S->sigma_prev);
    const GatherF32 gx{qc};
    ef::df dot{0.0f, 0.0f};
    for (uint32_t h = blockIdx.x; h < (1u << P.H); h += gridDim.x) {
        const int k = P.A - __popc(h);
        if (k < 0 || k > P.K) continue;
        __syncthreads();
        uint32_t off;
        const int n = blk_setup_block(P, tb, h, k, sh, &off);
        for (int r = threadIdx.x; r < n; r += blockDim.x) Xs[r] = gx(off + r);
        __syncthreads();
        for (int r = threadIdx.x; r < n; r += blockDim.x) {
            float acc[NC];
            int cnt[NC];
            blk_row<float, NC>(P, tb, k, off, r, sh.list[r], Xs, sh, gx, acc, cnt);
            const float hv = blk_y_f32<NC>(P, acc, cnt, Xs[r]);
            const float uu = sig * hv - gam * qp[off + r];
            qp[off + r] = uu;
            dot = ef::df_add(dot, ef::two_prod(sig * Xs[r], uu));
        }
    }
    const double d = block_sum<BLK_NT>((double)dot.hi + (double)dot.lo, red);
    if (threadIdx.x == 0) part[blockIdx.x] = d;
}

template <class K_t>
static int set_smem(K_t kern, size_t sm) {
    HM_CUDA(cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm));
    return HM_OK;
}

// Lanczos hooks: plan (0 = block path usable), attribute setup, launch
int blk_lz_plan(hm_basis *b, const BondParams &bp, int dtype, BlkParams *P, int *blocks) {
    int rc = blk_plan(b, bp, blk_K(b), P);
    if (rc != 0) return rc;
    const size_t sm = blk_smem_bytes(*P, dtype == HM_F64 ? 8 : 4, 1);
    if (sm > 227 * 1024) return 1;
    int per = 1;
    if (dtype == HM_F64) {
        if (P->nc == 1) { HM_TRY(set_smem(k_blk_lz64<1>, sm)); HM_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per, k_blk_lz64<1>, BLK_NT, sm)); }
        else if (P->nc == 2) { HM_TRY(set_smem(k_blk_lz64<2>, sm)); HM_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per, k_blk_lz64<2>, BLK_NT, sm)); }
        else { HM_TRY(set_smem(k_blk_lz64<4>, sm)); HM_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per, k_blk_lz64<4>, BLK_NT, sm)); }
    } else {
        if (P->nc == 1) { HM_TRY(set_smem(k_blk_lz32<1>, sm)); HM_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per, k_blk_lz32<1>, BLK_NT, sm)); }
        else if (P->nc == 2) { HM_TRY(set_smem(k_blk_lz32<2>, sm)); HM_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per, k_blk_lz32<2>, BLK_NT, sm)); }
        else { HM_TRY(set_smem(k_blk_lz32<4>, sm)); HM_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per, k_blk_lz32<4>, BLK_NT, sm)); }
    }
    *blocks = std::min<int>(sm_count() * std::max(per, 1), 1 << P->H);
    return 0;
}

int blk_lz64_launch(const BlkParams &P, const long long *Xc, const long long *Xp, unsigned long long *Y,
                    LzScalars *S, int pc, double *part, int blocks, cudaStream_t st) {
    const size_t sm = blk_smem_bytes(P, 8, 1);
    if (P.nc == 1) k_blk_lz64<1><<<blocks, BLK_NT, sm, st>>>(P, Xc, Xp, Y, S, pc, part);
    else if (P.nc == 2) k_blk_lz64<2><<<blocks, BLK_NT, sm, st>>>(P, Xc, Xp, Y, S, pc, part);
    else k_blk_lz64<4><<<blocks, BLK_NT, sm, st>>>(P, Xc, Xp, Y, S, pc, part);
    HM_CUDA(cudaGetLastError());
    return HM_OK;
}

int blk_lz32_launch(const BlkParams &P, const float *qc, float *qp, LzScalars *S, double *part, int blocks,
                    cudaStream_t st) {
    const size_t sm = blk_smem_bytes(P, 4, 1);
    if (P.nc == 1) k_blk_lz32<1><<<blocks, BLK_NT, sm, st>>>(P, qc, qp, S, part);
    else if (P.nc == 2) k_blk_lz32<2><<<blocks, BLK_NT, sm, st>>>(P, qc, qp, S, part);
    else k_blk_lz32<4><<<blocks, BLK_NT, sm, st>>>(P, qc, qp, S, part);
    HM_CUDA(cudaGetLastError());
    return HM_OK;
}

// returns 1 when the block path does not apply (caller falls back to the row kernel)
int blk_matvec(hm_basis *b, const BondParams &bp, const void *x, void *y, int dtype, int nvec,
               cudaStream_t st) {
    if (nvec != 1) return 1;
    BlkParams P;
    int rc = blk_plan(b, bp, blk_K(b), &P);
    if (rc != 0) return rc;
    if (blk_smem_bytes(P, dtype == HM_F64 ? 8 : 4, 1) > 227 * 1024) return 1;
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
