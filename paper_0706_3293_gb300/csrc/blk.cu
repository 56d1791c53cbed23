// blk.cu -- host planning and the matvec kernel of the s = 1/2 block path (blk.cuh).
#include <algorithm>
#include <climits>
#include <cstring>
#include <map>
#include <tuple>

#include "blk.cuh"

namespace hm {

constexpr int BLK_NT = 1024;

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
    // low groups keyed by (class, d, type); high and cross bonds by class
    std::map<std::tuple<int, int, int>, uint32_t> groups;
    std::vector<std::pair<int, int>> hi[HM_BLK_MAXC], cr[HM_BLK_MAXC];
    for (int t = 0; t < bp.nb; ++t) {
        const int p = bp.p[t], q = bp.q[t];  // p < q
        if (q < K) {
            const int type = q < 8 ? 0 : (p >= 8 ? 1 : 2);
            groups[std::make_tuple(bc[t], q - p, type)] |= 1u << p;
        } else if (p >= K) {
            hi[bc[t]].push_back({p - K, q - K});
        } else {
            cr[bc[t]].push_back({p, q - K});
        }
    }
    if ((int)groups.size() > HM_BLK_MAXG) return 1;
    int g = 0;
    for (int c = 0; c < P->nc; ++c) {
        P->lg_start[c] = g;
        for (auto &kv : groups)
            if (std::get<0>(kv.first) == c) {
                P->lg_mask[g] = kv.second;
                P->lg_d[g] = (uint8_t)std::get<1>(kv.first);
                P->lg_type[g] = (uint8_t)std::get<2>(kv.first);
                ++g;
            }
    }
    for (int c = P->nc; c <= HM_BLK_MAXC; ++c) P->lg_start[c] = g;
    P->nlg = g;
    int nh = 0, ncr = 0;
    for (int c = 0; c < P->nc; ++c) {
        P->hb_start[c] = nh;
        for (auto &e : hi[c]) { P->hb_p[nh] = (uint8_t)e.first; P->hb_q[nh] = (uint8_t)e.second; ++nh; }
        P->cb_start[c] = ncr;
        for (auto &e : cr[c]) { P->cb_p[ncr] = (uint8_t)e.first; P->cb_q[ncr] = (uint8_t)e.second; ++ncr; }
    }
    for (int c = P->nc; c <= HM_BLK_MAXC; ++c) { P->hb_start[c] = nh; P->cb_start[c] = ncr; }
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

// shared memory: tables | low words (uint16) | staged values | per-block hop lists
size_t blk_smem_bytes(const BlkParams &P, int stage_bytes_per_row, int nvec) {
    size_t o = al16(P.tab_bytes);
    o += al16((size_t)P.max_block * 2);
    o += al16((size_t)P.max_block * stage_bytes_per_row * nvec);
    o += al16(HM_BLK_MAXB * 4) * 2 + al16(HM_BLK_MAXB) * 2;
    return o;
}

// ---------------------------------------------------------------------------------------
// the kernel
// ---------------------------------------------------------------------------------------
template <class T> struct Stage;
template <> struct Stage<double> { using type = int64_t; };
template <> struct Stage<float> { using type = float; };

__device__ __forceinline__ uint32_t gosper8(uint32_t v) {   // next byte with the same popcount
    const uint32_t t = v | (v - 1);
    return (t + 1) | (((~t & (t + 1)) - 1) >> (__ffs(v)));
}

template <class T>
__device__ __forceinline__ typename Stage<T>::type stage_val(const T *x, uint32_t j, int E) {
    if constexpr (sizeof(T) == 8) {
        const unsigned long long bits = __ldg((const unsigned long long *)x + j);
        return ef::fix_from_bits(bits, E);
    } else {
        return __ldg(x + j);
    }
}

// Per-block setup, shared by every block kernel: computes the block offset, the hop
// lists and the low words, stages the block's own x.  Returns the row count n.
template <class T>
struct BlkBlock {
    uint32_t off;
    int k, n;
};

template <class T, int NC>
__device__ __forceinline__ void blk_setup(const BlkParams &P, const BlkTabs &tb, uint32_t h, int k,
                                          const T *__restrict__ x, int E, uint16_t *list,
                                          typename Stage<T>::type *Xs, int *hdelta, uint32_t *coff,
                                          int8_t *ck, uint8_t *cbq, uint32_t *off_out, int *n_out) {
    const uint32_t off = blk_off(P, tb, h, k);
    const int n = (int)tb.C[P.K * (P.A + 1) + k];
    for (int e = threadIdx.x; e < P.nhb; e += blockDim.x) {
        const int p = P.hb_p[e], q = P.hb_q[e];
        const bool valid = ((h >> p) ^ (h >> q)) & 1u;
        hdelta[e] = valid ? (int)(blk_off(P, tb, h ^ ((1u << p) | (1u << q)), k) - off) : INT_MIN;
    }
    for (int e = threadIdx.x; e < P.ncb; e += blockDim.x) {
        const int q = P.cb_q[e];
        const uint32_t bq = (h >> q) & 1u;
        const int k2 = k + (bq ? 1 : -1);
        const bool ok = k2 >= 0 && k2 <= P.K;
        cbq[e] = (uint8_t)bq;
        ck[e] = (int8_t)(ok ? k2 : -1);
        coff[e] = ok ? blk_off(P, tb, h ^ (1u << q), k2) : 0u;
    }
    for (int b1 = threadIdx.x; b1 < P.nb1; b1 += blockDim.x) {
        const int c0 = k - __popc(b1);
        if (c0 < 0 || c0 > 8) continue;
        int base = tb.U[k * P.nb1 + b1];
        uint32_t b0 = (1u << c0) - 1u;
        const uint32_t hib = (uint32_t)b1 << 8;
        if (c0 == 0) { list[base] = (uint16_t)hib; continue; }
        while (b0 < 256u) {
            list[base++] = (uint16_t)(hib | b0);
            b0 = gosper8(b0);
        }
    }
    for (int r = threadIdx.x; r < n; r += blockDim.x) Xs[r] = stage_val<T>(x, off + r, E);
    *off_out = off;
    *n_out = n;
}

// Hop sums of one row.  acc[c]: sum of x over the allowed exchanges of class c (fixed
// point in FP64 mode), cnt[c]: their number.
template <class T, int NC>
__device__ __forceinline__ void blk_row(const BlkParams &P, const BlkTabs &tb, int k, uint32_t off,
                                        int r, uint32_t l, const T *__restrict__ x, int E,
                                        const typename Stage<T>::type *Xs, const int *hdelta,
                                        const uint32_t *coff, const int8_t *ck, const uint8_t *cbq,
                                        typename Stage<T>::type *acc, int *cnt) {
    using S = typename Stage<T>::type;
    const uint32_t R0own = tb.R0[l & 255u];
    const uint32_t R1own = (uint32_t)r - R0own;
    const uint16_t *Uk = tb.U + k * P.nb1;
#pragma unroll
    for (int c = 0; c < NC; ++c) {
        S a = S(0);
        int m_cnt = 0;
        // exchanges among the low positions: targets in this block (shared memory)
        for (int g = P.lg_start[c]; g < P.lg_start[c + 1]; ++g) {
            const int d = P.lg_d[g];
            const int type = P.lg_type[g];
            const uint32_t pat = 1u | (1u << d);
            uint32_t m = ((l >> d) ^ l) & P.lg_mask[g];
            while (m) {
                const int p = __ffs(m) - 1;
                m &= m - 1;
                const uint32_t l2 = l ^ (pat << p);
                uint32_t r2;
                if (type == 0) r2 = R1own + tb.R0[l2 & 255u];
                else if (type == 1) r2 = R0own + Uk[l2 >> 8];
                else r2 = (uint32_t)Uk[l2 >> 8] + tb.R0[l2 & 255u];
                a += Xs[r2];
                ++m_cnt;
            }
        }
        // exchanges across the split: one bit flips on each side
        for (int e = P.cb_start[c]; e < P.cb_start[c + 1]; ++e) {
            const int p = P.cb_p[e];
            if ((((l >> p) & 1u) != cbq[e]) && ck[e] >= 0) {
                const uint32_t l2 = l ^ (1u << p);
                const uint32_t j = coff[e] + rank_low(P, tb, l2, ck[e]);
                a += stage_val<T>(x, j, E);
                ++m_cnt;
            }
        }
        // exchanges among the high positions: the same row of another block
        for (int e = P.hb_start[c]; e < P.hb_start[c + 1]; ++e) {
            const int dl = hdelta[e];
            if (dl != INT_MIN) {
                a += stage_val<T>(x, (uint32_t)((int)(off + (uint32_t)r) + dl), E);
                ++m_cnt;
            }
        }
        acc[c] = a;
        cnt[c] = m_cnt;
    }
}

// y_i from the class sums: sum_c (-J_c/4) (2 acc_c + (ntot_c - 2 cnt_c) x_i)
template <int NC>
__device__ __forceinline__ ef::df blk_combine_f64(const BlkParams &P, const int64_t *acc, const int *cnt,
                                                  int64_t Xo, int E, int scale) {
    ef::df y{0.0f, 0.0f};
#pragma unroll
    for (int c = 0; c < NC; ++c) {
        const int64_t Tc = 2 * acc[c] + (int64_t)(P.ntot[c] - 2 * cnt[c]) * Xo;
        const ef::df t = ef::df_from_fix(Tc, E, 0, scale);
        y = ef::df_add(y, ef::df_mul(t, ef::df{P.g_hi[c], P.g_lo[c]}));
    }
    return y;
}

template <int NC>
__device__ __forceinline__ float blk_combine_f32(const BlkParams &P, const float *acc, const int *cnt, float xo) {
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

template <class T, int NC>
__global__ void __launch_bounds__(BLK_NT, 1)
k_blk_matvec(BlkParams P, const T *__restrict__ x, T *__restrict__ y, const int *__restrict__ Eptr) {
    using S = typename Stage<T>::type;
    extern __shared__ __align__(16) unsigned char smem[];
    const BlkTabs tb = stage_blk_tables(P, smem);
    size_t o = al16(P.tab_bytes);
    uint16_t *list = (uint16_t *)(smem + o); o += al16((size_t)P.max_block * 2);
    S *Xs = (S *)(smem + o); o += al16((size_t)P.max_block * sizeof(S));
    int *hdelta = (int *)(smem + o); o += al16(HM_BLK_MAXB * 4);
    uint32_t *coff = (uint32_t *)(smem + o); o += al16(HM_BLK_MAXB * 4);
    int8_t *ck = (int8_t *)(smem + o); o += al16(HM_BLK_MAXB);
    uint8_t *cbq = (uint8_t *)(smem + o);
    const int E = Eptr ? *Eptr : 0;
    const int scale = E - 1023;
    for (uint32_t h = blockIdx.x; h < (1u << P.H); h += gridDim.x) {
        const int k = P.A - __popc(h);
        if (k < 0 || k > P.K) continue;
        __syncthreads();    // previous block done with the shared buffers
        uint32_t off;
        int n;
        blk_setup<T, NC>(P, tb, h, k, x, E, list, Xs, hdelta, coff, ck, cbq, &off, &n);
        __syncthreads();
        for (int r = threadIdx.x; r < n; r += blockDim.x) {
            const uint32_t l = list[r];
            S acc[NC];
            int cnt[NC];
            blk_row<T, NC>(P, tb, k, off, r, l, x, E, Xs, hdelta, coff, ck, cbq, acc, cnt);
            if constexpr (sizeof(T) == 8) {
                const ef::df v = blk_combine_f64<NC>(P, acc, cnt, Xs[r], E, scale);
                ((unsigned long long *)y)[off + r] = ef::bits_from_df(v, scale);
            } else {
                y[off + r] = blk_combine_f32<NC>(P, acc, cnt, Xs[r]);
            }
        }
    }
}

template <class T, int NC>
static int launch_blk_matvec(hm_basis *b, const BlkParams &P, const T *x, T *y, cudaStream_t st) {
    const size_t sm = blk_smem_bytes(P, sizeof(typename Stage<T>::type), 1);
    HM_CUDA(cudaFuncSetAttribute(k_blk_matvec<T, NC>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm));
    int *Ed = nullptr;
    if constexpr (sizeof(T) == 8) {
        Ed = (int *)b->d_scratch;
        HM_CUDA(cudaMemsetAsync(Ed, 0, sizeof(int), st));
        k_max_exp<<<grid_blocks(P.dim, 256), 256, 0, st>>>((const unsigned long long *)x, P.dim, Ed);
        HM_CUDA(cudaGetLastError());
    }
    const int blocks = std::min<int>(sm_count(), 1 << P.H);
    k_blk_matvec<T, NC><<<blocks, BLK_NT, sm, st>>>(P, x, y, Ed);
    HM_CUDA(cudaGetLastError());
    return HM_OK;
}

// ---------------------------------------------------------------------------------------
// Lanczos product: u = sigma_cur H q_cur - beta_prev sigma_prev q_prev, written over
// q_prev; part[blockIdx] = sum_i (sigma_cur q_cur,i) u_i.  Buffer parity pc holds q_cur.
// FP64: the row result, u and the dot are double-float; no FP64 instruction per row.
// ---------------------------------------------------------------------------------------
__device__ __forceinline__ ef::df df_of_double(double v) {
    const float hi = (float)v;
    return ef::df{hi, (float)(v - (double)hi)};
}

template <class T, int NC>
__global__ void __launch_bounds__(BLK_NT, 1)
k_blk_lz(BlkParams P, const T *__restrict__ qc, T *__restrict__ qp, LzScalars *S, int pc,
         double *__restrict__ part) {
    using S_t = typename Stage<T>::type;
    if (S->done) return;
    extern __shared__ __align__(16) unsigned char smem[];
    __shared__ double red[BLK_NT / 32];
    const BlkTabs tb = stage_blk_tables(P, smem);
    size_t o = al16(P.tab_bytes);
    uint16_t *list = (uint16_t *)(smem + o); o += al16((size_t)P.max_block * 2);
    S_t *Xs = (S_t *)(smem + o); o += al16((size_t)P.max_block * sizeof(S_t));
    int *hdelta = (int *)(smem + o); o += al16(HM_BLK_MAXB * 4);
    uint32_t *coff = (uint32_t *)(smem + o); o += al16(HM_BLK_MAXB * 4);
    int8_t *ck = (int8_t *)(smem + o); o += al16(HM_BLK_MAXB);
    uint8_t *cbq = (uint8_t *)(smem + o);
    const int E = S->emax[pc];
    const int Ep = S->emax[pc ^ 1];
    const int scale = E - 1023, scale_p = Ep - 1023;
    // per-thread copies of the step scalars (a few FP64 operations per thread, not per row)
    const ef::df sig_s = df_of_double(ldexp(S->sigma_cur, scale));
    const ef::df gam_s = df_of_double(ldexp(S->beta_prev * S->sigma_prev, scale_p));
    const float sig_f = (float)S->sigma_cur, gam_f = (float)(S->beta_prev * S->sigma_prev);
    ef::df dot{0.0f, 0.0f};
    for (uint32_t h = blockIdx.x; h < (1u << P.H); h += gridDim.x) {
        const int k = P.A - __popc(h);
        if (k < 0 || k > P.K) continue;
        __syncthreads();
        uint32_t off;
        int n;
        blk_setup<T, NC>(P, tb, h, k, qc, E, list, Xs, hdelta, coff, ck, cbq, &off, &n);
        __syncthreads();
        for (int r = threadIdx.x; r < n; r += blockDim.x) {
            const uint32_t l = list[r];
            S_t acc[NC];
            int cnt[NC];
            blk_row<T, NC>(P, tb, k, off, r, l, qc, E, Xs, hdelta, coff, ck, cbq, acc, cnt);
            if constexpr (sizeof(T) == 8) {
                // H q in units of 2^scale (the vector's own scale), then
                // u = (sigma 2^scale) hv - (gamma 2^scale_p) (q_prev 2^-scale_p)
                const ef::df hv = blk_combine_f64<NC>(P, acc, cnt, Xs[r], E, scale);
                const unsigned long long pb = ((const unsigned long long *)qp)[off + r];
                const ef::df qpv = ef::df_from_bits(pb, scale_p);
                const ef::df u = ef::df_add(ef::df_mul(sig_s, hv), ef::df_neg(ef::df_mul(gam_s, qpv)));
                ((unsigned long long *)qp)[off + r] = ef::bits_from_df(u, 0);
                const ef::df v = ef::df_mul(sig_s, ef::df_from_fix(Xs[r], E, 0, scale));
                dot = ef::df_add(dot, ef::df_mul(v, u));
            } else {
                const float hv = blk_combine_f32<NC>(P, acc, cnt, Xs[r]);
                const float u = sig_f * hv - gam_f * qp[off + r];
                qp[off + r] = u;
                dot = ef::df_add(dot, ef::two_prod(sig_f * Xs[r], u));
            }
        }
    }
    double d = block_sum<BLK_NT>((double)dot.hi + (double)dot.lo, red);
    if (threadIdx.x == 0) part[blockIdx.x] = d;
}

template <class T, int NC>
static int launch_blk_lz(const BlkParams &P, const T *qc, T *qp, LzScalars *S, int pc, double *part,
                         int blocks, cudaStream_t st) {
    const size_t sm = blk_smem_bytes(P, sizeof(typename Stage<T>::type), 1);
    k_blk_lz<T, NC><<<blocks, BLK_NT, sm, st>>>(P, qc, qp, S, pc, part);
    HM_CUDA(cudaGetLastError());
    return HM_OK;
}

template <class T, int NC>
static int prep_blk_lz(const BlkParams &P) {
    const size_t sm = blk_smem_bytes(P, sizeof(typename Stage<T>::type), 1);
    HM_CUDA(cudaFuncSetAttribute(k_blk_lz<T, NC>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm));
    return HM_OK;
}

// Lanczos hooks: plan (0 = block path usable), attribute setup, launch
int blk_lz_plan(hm_basis *b, const BondParams &bp, int dtype, BlkParams *P, int *blocks) {
    int rc = blk_plan(b, bp, 16, P);
    if (rc != 0) return rc;
    const size_t stage = dtype == HM_F64 ? 8 : 4;
    if (blk_smem_bytes(*P, (int)stage, 1) > 227 * 1024) return 1;
    *blocks = std::min<int>(sm_count(), 1 << P->H);
    if (dtype == HM_F64) {
        if (P->nc == 1) return prep_blk_lz<double, 1>(*P);
        if (P->nc == 2) return prep_blk_lz<double, 2>(*P);
        return prep_blk_lz<double, 4>(*P);
    }
    if (P->nc == 1) return prep_blk_lz<float, 1>(*P);
    if (P->nc == 2) return prep_blk_lz<float, 2>(*P);
    return prep_blk_lz<float, 4>(*P);
}

int blk_lz_launch(const BlkParams &P, int dtype, const void *qc, void *qp, LzScalars *S, int pc,
                  double *part, int blocks, cudaStream_t st) {
    if (dtype == HM_F64) {
        if (P.nc == 1) return launch_blk_lz<double, 1>(P, (const double *)qc, (double *)qp, S, pc, part, blocks, st);
        if (P.nc == 2) return launch_blk_lz<double, 2>(P, (const double *)qc, (double *)qp, S, pc, part, blocks, st);
        return launch_blk_lz<double, 4>(P, (const double *)qc, (double *)qp, S, pc, part, blocks, st);
    }
    if (P.nc == 1) return launch_blk_lz<float, 1>(P, (const float *)qc, (float *)qp, S, pc, part, blocks, st);
    if (P.nc == 2) return launch_blk_lz<float, 2>(P, (const float *)qc, (float *)qp, S, pc, part, blocks, st);
    return launch_blk_lz<float, 4>(P, (const float *)qc, (float *)qp, S, pc, part, blocks, st);
}

// returns 1 when the block path does not apply (caller falls back to the row kernel)
int blk_matvec(hm_basis *b, const BondParams &bp, const void *x, void *y, int dtype, int nvec,
               cudaStream_t st) {
    if (nvec != 1) return 1;
    BlkParams P;
    int rc = blk_plan(b, bp, 16, &P);
    if (rc != 0) return rc;
    const size_t stage = dtype == HM_F64 ? 8 : 4;
    if (blk_smem_bytes(P, (int)stage, 1) > 227 * 1024) return 1;
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
