// s1blk.cu -- block-structured products for s = 1 sectors (layout in s1_sweep.cuh).
//
// As on the s = 1/2 block path (blk.cuh):
//   * a CTA stages its block's x in shared memory; exchanges among low sites gather there;
//   * exchanges among high sites keep the low word, so they gather the same row of another
//     block (coalesced), its offset encoded once per block;
//   * exchanges across the split read one other block, shared by all rows of the block.
// The kernels specialised to the bond list at run time (jit.cu, bodies in s1_sweep.cuh)
// read the exchange targets among the low words from the rank tables rl / rx; the generic
// kernel below (the fallback without NVRTC, HM_JIT=0) walks its bond lists at run time and
// re-encodes every target word with the rank table of all packed low words.
#include <algorithm>
#include <cmath>
#include <cstdlib>
#include <vector>

#include "ef64.cuh"
#include "s1blk.cuh"

namespace hm {

// Every block through rowf(r, l, x_r, y_r) after its set-up; LZ: Lanczos product
// u = sigma H q - gamma q_prev written over q_prev and part[block] = sum (sigma q . u)
template <bool LZ>
__device__ __forceinline__ void s1_body(const S1Plan &P, const float *__restrict__ x, float *__restrict__ y,
                                        const LzScalars *__restrict__ S, double *__restrict__ part) {
    if (LZ && S->done) return;
    extern __shared__ __align__(16) unsigned char smem[];
    uint32_t *cd = (uint32_t *)smem;                                   // [cd_len]
    float *Xs = (float *)(smem + ((P.cd_len * 4 + 15) & ~15));         // [max_block]
    __shared__ uint32_t s_hoff[2 * S1_MAXB];      // high exchange (bond, direction): target block or ~0
    __shared__ uint32_t s_cb[2 * S1_MAXB];        // cross exchange (bond, direction): target block or ~0
    __shared__ float s_cm[S1_MAXB];               // cross bond: m of its high site in this block
    __shared__ float s_bdiag;
    __shared__ double red[S1_NT / 32];
    const int tid = threadIdx.x;
    for (int i = tid; i < P.cd_len; i += S1_NT) cd[i] = P.cd[i];
    const float sg = LZ ? (float)S->sigma_cur : 1.0f, gm = LZ ? (float)(S->beta_prev * S->sigma_prev) : 0.0f;
    __syncthreads();
    for (int bi = blockIdx.x; bi < P.nblocks; bi += gridDim.x) {
        const uint4 bk = P.blocks[bi];
        const uint32_t h = bk.x, off = bk.y;
        const int k = (int)bk.z, n = (int)bk.w;
        // set-up: neighbouring blocks of the high and cross exchanges, the high-site diagonal
        if (tid < 2 * P.nhi) {
            const int j = tid >> 1, d = tid & 1, p = P.hi_p[j], q = P.hi_q[j];
            const int ap = s1_dig(h, p), aq = s1_dig(h, q);
            const bool ok = d == 0 ? (ap >= 1 && aq <= 1) : (ap <= 1 && aq >= 1);
            const uint32_t h2 = d == 0 ? h - (1u << (2 * p)) + (1u << (2 * q)) : h + (1u << (2 * p)) - (1u << (2 * q));
            s_hoff[tid] = ok ? s1_off(P, cd, h2, k) : 0xFFFFFFFFu;
        } else if (tid >= 256 && tid < 256 + 2 * P.ncr) {
            const int e = tid - 256, j = e >> 1, d = e & 1, q = P.cr_q[j];
            const int aq = s1_dig(h, q);
            // d = 0: the low site gives a unit to the high site (k - 1); d = 1: the reverse
            const int k2 = d == 0 ? k - 1 : k + 1;
            const bool ok = (d == 0 ? aq <= 1 : aq >= 1) && k2 >= 0 && k2 <= 2 * P.K;
            const uint32_t h2 = d == 0 ? h + (1u << (2 * q)) : h - (1u << (2 * q));
            s_cb[e] = ok ? s1_off(P, cd, h2, k2) : 0xFFFFFFFFu;
            if (d == 0) s_cm[j] = (float)(1 - aq);
        }
        if (tid == S1_NT - 1) {
            float dsum = 0.0f;
            for (int j = 0; j < P.nhi; ++j)
                dsum += P.hi_j[j] * (float)((1 - s1_dig(h, P.hi_p[j])) * (1 - s1_dig(h, P.hi_q[j])));
            s_bdiag = dsum;
        }
        for (int r = tid; r < n; r += S1_NT) Xs[r] = x[off + r];
        __syncthreads();
        const uint32_t *lwk = P.lw + P.lwoff[k];
        ef::df dot{0.0f, 0.0f};
        for (int r = tid; r < n; r += S1_NT) {
            const uint32_t l = __ldg(lwk + r);
            const float xo = Xs[r];
            float dg = s_bdiag, acc = 0.0f;
            for (int j = 0; j < P.nlo; ++j) {
                const int p = P.lo_p[j], q = P.lo_q[j];
                const int ap = s1_dig(l, p), aq = s1_dig(l, q);
                const float Jm = P.lo_j[j];
                dg += Jm * (float)((1 - ap) * (1 - aq));
                if (ap >= 1 && aq <= 1) acc += Jm * Xs[__ldg(P.lut + (l - (1u << (2 * p)) + (1u << (2 * q))))];
                if (ap <= 1 && aq >= 1) acc += Jm * Xs[__ldg(P.lut + (l + (1u << (2 * p)) - (1u << (2 * q))))];
            }
            for (int j = 0; j < P.ncr; ++j) {
                const int p = P.cr_p[j];
                const int ap = s1_dig(l, p);
                const float Jm = P.cr_j[j];
                dg += Jm * (float)(1 - ap) * s_cm[j];
                const uint32_t b0 = s_cb[2 * j], b1 = s_cb[2 * j + 1];
                if (b0 != 0xFFFFFFFFu && ap >= 1) acc += Jm * __ldg(x + b0 + __ldg(P.lut + (l - (1u << (2 * p)))));
                if (b1 != 0xFFFFFFFFu && ap <= 1) acc += Jm * __ldg(x + b1 + __ldg(P.lut + (l + (1u << (2 * p)))));
            }
            for (int e = 0; e < 2 * P.nhi; ++e) {
                const uint32_t t = s_hoff[e];
                if (t != 0xFFFFFFFFu) acc += P.hi_j[e >> 1] * __ldg(x + t + r);
            }
            const float hv = dg * xo + acc;
            if constexpr (LZ) {
                const float u = sg * hv - gm * y[off + r];
                y[off + r] = u;
                dot = ef::df_add(dot, ef::two_prod(sg * xo, u));
            } else {
                y[off + r] = hv;
            }
        }
        if constexpr (LZ) {
            const double t = block_sum<S1_NT>((double)dot.hi + (double)dot.lo, red);
            if (tid == 0) part[bi] = t;
        }
        __syncthreads();                 // the shared set-up of the next block overwrites this one's
    }
}

__global__ void __launch_bounds__(S1_NT) k_s1_mv(S1Plan P, const float *__restrict__ x, float *__restrict__ y) {
    s1_body<false>(P, x, y, nullptr, nullptr);
}
__global__ void __launch_bounds__(S1_NT) k_s1_lz32(S1Plan P, const float *__restrict__ qc, float *__restrict__ qp,
                                                  const LzScalars *__restrict__ S, double *__restrict__ part) {
    s1_body<true>(P, qc, qp, S, part);
}

// ---- host -------------------------------------------------------------------------------------

static int s1_tables(hm_basis *b, int K, S1Tab *out) {
    const SectorView &sv = b->view;
    const int N = sv.N, H = N - K, A = sv.A, W = 2 * N + 1;
    auto D = [&](int sites, int a) -> uint64_t { return a < 0 || a > 2 * sites ? 0 : b->D[(size_t)sites * W + a]; };
    auto CD = [&](int p, int S, int a) -> uint64_t { return b->cd[(size_t)p * sv.cd_rowlen + (size_t)S * sv.cd_w + a]; };
    // low words: rank_K by the Sec. 3.2 sums over positions 1..K-1
    const size_t nlut = (size_t)1 << (2 * K);
    std::vector<uint16_t> lut(nlut, 0);
    std::vector<int> lwoff(2 * K + 2, 0);
    for (int k = 0; k <= 2 * K; ++k) lwoff[k + 1] = lwoff[k] + (int)D(K, k);
    std::vector<uint32_t> lw(lwoff[2 * K + 1]);
    for (size_t w = 0; w < nlut; ++w) {
        int S = 0;
        uint64_t r = 0;
        bool ok = true;
        for (int p = 0; p < K; ++p) {
            const int a = (int)((w >> (2 * p)) & 3);
            S += a;
            if (a > 2 || S > A) { ok = false; break; }     // not a digit / beyond the table's sums
            if (p >= 1) r += CD(p, S, a);
        }
        if (!ok || S > A) continue;
        lut[w] = (uint16_t)r;
        lw[lwoff[S] + r] = (uint32_t)w;
    }
    // blocks: every high word whose low part can hold the rest of the digit sum, in row order
    std::vector<uint4> blocks;
    const uint64_t nh = 1;
    uint64_t nhigh = nh;
    for (int t = 0; t < H; ++t) nhigh *= 3;
    int mb = 0;
    for (uint64_t c = 0; c < nhigh; ++c) {
        uint32_t h = 0;
        int sum = 0;
        uint64_t cc = c;
        for (int t = 0; t < H; ++t) { const int a = (int)(cc % 3); cc /= 3; h |= (uint32_t)a << (2 * t); sum += a; }
        const int k = A - sum;
        if (k < 0 || k > 2 * K) continue;
        uint64_t off = 0;
        int S = k;
        for (int t = 0; t < H; ++t) { const int a = (int)((h >> (2 * t)) & 3); S += a; off += CD(K + t, S, a); }
        const int n = lwoff[k + 1] - lwoff[k];
        blocks.push_back(make_uint4(h, (uint32_t)off, (uint32_t)k, (uint32_t)n));
        mb = std::max(mb, n);
    }
    std::sort(blocks.begin(), blocks.end(), [](const uint4 &x, const uint4 &y) { return x.y < y.y; });
    // exchange rank tables of the low words: rl[pi nlw + g] for the site pair
    // pi = q (q - 1) / 2 + p (p < q), rx[p nlw + g]; direction d in the low (d = 0) or high
    // (d = 1) 16 bits, 0xFFFF where not allowed.
    // Only the digit sums kmin..kmax of the sector's blocks have ranks (the CD table of
    // the sector holds no others); every entry is checked to be a row of the class it
    // addresses.
    const int nlw = lwoff[2 * K + 1], kmax = std::min(A, 2 * K), kmin = std::max(0, A - 2 * H);
    const int npair = K * (K - 1) / 2;
    for (int k = 0; k <= 2 * K; ++k)
        if (D(K, k) >= 0xFFFF) return 1;               // ranks and the 0xFFFF mark share 16 bits
    std::vector<uint32_t> rl((size_t)npair * nlw, 0xFFFFFFFFu), rx((size_t)K * nlw, 0xFFFFFFFFu);
    auto put_rank = [](uint32_t &e, int d, uint16_t v) {
        e = d == 0 ? (e & 0xFFFF0000u) | v : (e & 0xFFFFu) | ((uint32_t)v << 16);
    };
    bool bad = false;
    auto rank_of = [&](uint32_t w, int k2) -> uint16_t {
        const uint16_t v = lut[w];
        if (k2 < kmin || k2 > kmax || (uint64_t)v >= D(K, k2)) bad = true;
        return v;
    };
    for (int k = kmin; k <= kmax; ++k)
        for (int g = lwoff[k]; g < lwoff[k + 1]; ++g) {
            const uint32_t l = lw[g];
            for (int p = 0; p < K; ++p) {
                const int ap = (int)((l >> (2 * p)) & 3);
                uint32_t &ex = rx[(size_t)p * nlw + g];
                if (ap >= 1 && k - 1 >= kmin) put_rank(ex, 0, rank_of(l - (1u << (2 * p)), k - 1));
                if (ap <= 1 && k + 1 <= kmax) put_rank(ex, 1, rank_of(l + (1u << (2 * p)), k + 1));
                for (int q = p + 1; q < K; ++q) {
                    const int aq = (int)((l >> (2 * q)) & 3), pi = q * (q - 1) / 2 + p;
                    uint32_t &el = rl[(size_t)pi * nlw + g];
                    if (ap >= 1 && aq <= 1) put_rank(el, 0, rank_of(l - (1u << (2 * p)) + (1u << (2 * q)), k));
                    if (ap <= 1 && aq >= 1) put_rank(el, 1, rank_of(l + (1u << (2 * p)) - (1u << (2 * q)), k));
                }
            }
        }
    if (bad) return 1;                                 // not used: the general kernel serves
    auto al = [](size_t x) { return (x + 255) & ~(size_t)255; };
    const size_t b_lut = al(nlut * 2), b_lw = al(lw.size() * 4), b_bl = al(blocks.size() * sizeof(uint4));
    const size_t b_rl = al(rl.size() * 4), b_rx = al(rx.size() * 4);
    const size_t bytes = b_lut + b_lw + b_bl + b_rl + b_rx;
    unsigned char *dev = nullptr;
    HM_CUDA(cudaMalloc(&dev, bytes));
    HM_CUDA(cudaMemcpy(dev, lut.data(), nlut * 2, cudaMemcpyHostToDevice));
    HM_CUDA(cudaMemcpy(dev + b_lut, lw.data(), lw.size() * 4, cudaMemcpyHostToDevice));
    HM_CUDA(cudaMemcpy(dev + b_lut + b_lw, blocks.data(), blocks.size() * sizeof(uint4), cudaMemcpyHostToDevice));
    if (!rl.empty()) HM_CUDA(cudaMemcpy(dev + b_lut + b_lw + b_bl, rl.data(), rl.size() * 4, cudaMemcpyHostToDevice));
    HM_CUDA(cudaMemcpy(dev + b_lut + b_lw + b_bl + b_rl, rx.data(), rx.size() * 4, cudaMemcpyHostToDevice));
    out->dev = dev;
    out->lut = (uint16_t *)dev;
    out->lw = (uint32_t *)(dev + b_lut);
    out->blocks = (uint4 *)(dev + b_lut + b_lw);
    out->rl = (uint32_t *)(dev + b_lut + b_lw + b_bl);
    out->rx = (uint32_t *)(dev + b_lut + b_lw + b_bl + b_rl);
    out->nlw = nlw;
    out->nblocks = (int)blocks.size();
    out->max_block = mb;
    out->K = K;
    for (int k = 0; k <= 2 * K + 1; ++k) out->lwoff[k] = lwoff[k];
    return HM_OK;
}

// split of the s = 1 block path: K = min(10, N - 2) low sites
static int s1_K(const hm_basis *b) { return std::min(S1_KMAX, b->view.N - 2); }

// plan of the s = 1 block path; 1 when it does not apply (caller: the general row kernel)
int s1_plan(hm_basis *b, const BondParams &bp, S1Plan *P) {
    const SectorView &sv = b->view;
    if (sv.S2 != 2 || sv.idx64 || b->parity || sv.N < 6 || sv.N > 24) return 1;
    const int K = s1_K(b), H = sv.N - K;
    if (2 * H > 32) return 1;
    // s = 1: every exchange factor 1/2 sqrt(radicands) is 1 (checked, not assumed)
    for (int ap = 0; ap <= 2; ++ap)
        for (int aq = 0; aq <= 2; ++aq) {
            if (ap >= 1 && aq <= 1 && std::fabs(bp.hs_pdn[ap * 8 + aq] - 1.0) > 1e-15) return 1;
            if (ap <= 1 && aq >= 1 && std::fabs(bp.hs_pup[ap * 8 + aq] - 1.0) > 1e-15) return 1;
        }
    memset(P, 0, sizeof *P);
    for (int t = 0; t < bp.nb; ++t) {
        const int p = bp.p[t], q = bp.q[t];       // p < q
        const float j = (float)bp.jm[t];
        if (q < K) {
            if (P->nlo == S1_MAXB) return 1;
            P->lo_p[P->nlo] = (uint8_t)p; P->lo_q[P->nlo] = (uint8_t)q; P->lo_j[P->nlo++] = j;
        } else if (p >= K) {
            if (P->nhi == S1_MAXB) return 1;
            P->hi_p[P->nhi] = (uint8_t)(p - K); P->hi_q[P->nhi] = (uint8_t)(q - K); P->hi_j[P->nhi++] = j;
        } else {
            if (P->ncr == S1_MAXB) return 1;
            P->cr_p[P->ncr] = (uint8_t)p; P->cr_q[P->ncr] = (uint8_t)(q - K); P->cr_j[P->ncr++] = j;
        }
    }
    auto it = b->s1_tabs.find(K);
    if (it == b->s1_tabs.end()) {
        S1Tab t;
        const int rc = s1_tables(b, K, &t);
        if (rc != 0) return rc;
        it = b->s1_tabs.emplace(K, t).first;
    }
    const S1Tab &T = it->second;
    P->N = sv.N; P->K = K; P->H = H; P->A = sv.A;
    P->nblocks = T.nblocks; P->max_block = T.max_block;
    P->lut = T.lut; P->lw = T.lw; P->blocks = T.blocks;
    P->nlw = T.nlw; P->rl = T.rl; P->rx = T.rx;
    // FP64 couplings: C_b = round(-J_b 2^cs) with max |J_b| 2^cs < 2^52, so |C_b| <= 2^52
    // (the split products of s1_mac) and every row's diagonal sum fits in int64
    double maxj = 0.0;
    for (int t = 0; t < bp.nb; ++t) maxj = std::max(maxj, std::fabs(bp.jm[t]));
    int e2 = 0;
    if (maxj > 0.0) std::frexp(maxj, &e2);            // maxj < 2^e2
    P->cs = 52 - e2;
    auto cfix = [&](double jm) { return (long long)std::llround(std::ldexp(jm, P->cs)); };
    {
        int il = 0, ih = 0, ic = 0;
        for (int t = 0; t < bp.nb; ++t) {
            const int p = bp.p[t], q = bp.q[t];
            if (q < K) P->lo_c[il++] = cfix(bp.jm[t]);
            else if (p >= K) P->hi_c[ih++] = cfix(bp.jm[t]);
            else P->cr_c[ic++] = cfix(bp.jm[t]);
        }
    }
    P->cd = (const uint32_t *)sv.cd; P->cd_w = sv.cd_w; P->cd_rowlen = sv.cd_rowlen; P->cd_len = sv.cd_len;
    for (int k = 0; k <= 2 * K + 1; ++k) P->lwoff[k] = T.lwoff[k];
    const size_t sm = ((size_t)(P->cd_len * 4 + 15) & ~(size_t)15) + (size_t)P->max_block * 4;
    if (sm > 160 * 1024) return 1;
    return 0;
}

uint64_t s1_block_count(const hm_basis *b) {
    const SectorView &sv = b->view;
    if (sv.S2 != 2 || sv.idx64 || b->parity || sv.N < 6 || sv.N > 24) return 0;
    const int K = s1_K(b), H = sv.N - K, W = 2 * sv.N + 1;
    uint64_t n = 0;                  // high words of digit sum s: D(H, s) (trinomial)
    for (int s = 0; s <= 2 * H; ++s)
        if (sv.A - s >= 0 && sv.A - s <= 2 * K) n += b->D[(size_t)H * W + s];
    return n;
}

static size_t s1_smem(const S1Plan &P, int es) {
    return ((size_t)(P.cd_len * 4 + 15) & ~(size_t)15) + (size_t)P.max_block * es;
}

static int s1_grid(const S1Plan &P, const void *kern, size_t sm) {
    int per = 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per, kern, S1_NT, sm) != cudaSuccess) {
        cudaGetLastError();
        per = 1;
    }
    return std::max(1, std::min(sm_count() * std::max(per, 1), P.nblocks));
}

// the kernel of plan P specialised to its bonds (mode as in jit_s1_kernel), or nullptr
// when NVRTC cannot serve or HM_JIT=0 asks for the generic kernels
static const void *s1_jit(const S1Plan &P, int mode) {
    const char *e = getenv("HM_JIT");
    if (e && e[0] == '0') return nullptr;
    const void *k = nullptr;
    return jit_s1_kernel(P, mode, &k) == 0 ? k : nullptr;
}

static int s1_launch(const void *kern, const S1Plan &P, size_t sm, void **args, cudaStream_t st) {
    HM_CUDA(raise_smem_limit(kern, (int)sm));
    HM_CUDA(cudaLaunchKernel(kern, dim3(s1_grid(P, kern, sm)), dim3(S1_NT), args, sm, st));
    return HM_OK;
}

// y = H x, FP32, one vector
int s1_matvec(const S1Plan &P, const float *x, float *y, cudaStream_t st) {
    const void *k = s1_jit(P, 0);
    if (!k) k = (const void *)k_s1_mv;
    void *args[] = {(void *)&P, (void *)&x, (void *)&y};
    return s1_launch(k, P, s1_smem(P, 4), args, st);
}

// Lanczos product, FP32: q_prev <- sigma H q - gamma q_prev, part[block] = (sigma q . u) per block
int s1_lz32(const S1Plan &P, const float *qc, float *qp, const LzScalars *S, double *part, cudaStream_t st) {
    const void *k = s1_jit(P, 1);
    if (!k) k = (const void *)k_s1_lz32;
    void *args[] = {(void *)&P, (void *)&qc, (void *)&qp, (void *)&S, (void *)&part};
    return s1_launch(k, P, s1_smem(P, 4), args, st);
}

bool s1_jit_ready(const S1Plan &P, int mode) {
    if (mode == 2 && s1_smem(P, 8) > 200 * 1024) return false;
    return s1_jit(P, mode) != nullptr;
}

// Lanczos product, FP64 (specialised kernel only): Y = H q, part[block] = (q . y)
int s1_lz64(const S1Plan &P, const long long *Xc, unsigned long long *Y, const LzScalars *S, int pc, double *part,
            cudaStream_t st) {
    const void *k = s1_smem(P, 8) > 200 * 1024 ? nullptr : s1_jit(P, 2);
    if (!k) return fail(HM_EINVAL, "the FP64 s = 1 product needs its run-time compiled kernel");
    void *args[] = {(void *)&P, (void *)&Xc, (void *)&Y, (void *)&S, (void *)&pc, (void *)&part};
    return s1_launch(k, P, s1_smem(P, 8), args, st);
}

const char *s1_kernel_name(const S1Plan &P, int mode) {
    const bool j = s1_jit(P, mode) != nullptr;
    if (mode == 0) return j ? "k_s1_mv_jit" : "k_s1_mv";
    if (mode == 1) return j ? "k_s1_lz32_jit" : "k_s1_lz32";
    return j ? "k_s1_lz64_jit" : "none";
}

}  // namespace hm
