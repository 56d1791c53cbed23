// hm_internal.cuh -- shared definitions of libhm.so (not part of the C ABI).
//
// Sector tables, bond parameters, error reporting, the device codec (Sec. 3.1/3.2 of
// Schnack, Hage, Schmidt) and deterministic block reductions.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include <map>
#include <string>
#include <vector>

#include "../../include/hm.h"
#include "hm_dev.cuh"

// ---------------------------------------------------------------------------------------
// error reporting (thread-local message, see hm_last_error)
// ---------------------------------------------------------------------------------------
namespace hm {
int fail(int code, const char *fmt, ...);   // records the message, returns code
int cuda_fail(cudaError_t e, const char *what);
}  // namespace hm

#define HM_CUDA(call)                                                      \
    do {                                                                   \
        cudaError_t e_ = (call);                                           \
        if (e_ != cudaSuccess) return hm::cuda_fail(e_, #call);            \
    } while (0)

#define HM_TRY(call)                                                       \
    do {                                                                   \
        int rc_ = (call);                                                  \
        if (rc_ < 0) return rc_;                                           \
    } while (0)

// ---------------------------------------------------------------------------------------
// sector tables
// ---------------------------------------------------------------------------------------
namespace hm {
// CD[p][S][a] = sum_{n<a} D(p, S - n) for positions p = 0..N-1, prefix digit sums
// S = 0..A and digits a = 0..2s+1 (the last entry is the total D(p+1, S)).  With
// S_p = a_0 + ... + a_p, the 0-based index of a state is sum_{p>=1} CD[p][S_p][a_p]
// (Sec. 3.2), and decode walks p = N-1..1 choosing the digit whose cumulative range
// holds the residual index (Sec. 3.1).
struct SectorView {
    int N, S2, A, bits;     // bits per digit: 1, 2 or 4
    int cd_w;               // S2 + 2
    int cd_rowlen;          // (A + 1) * (S2 + 2)
    int cd_len;             // N * cd_rowlen
    int idx64;              // 1 when dim >= 2^32 (64-bit index arithmetic)
    uint64_t dim;
    const void *cd;         // device table, uint32_t (idx64 = 0) or uint64_t
};

}  // namespace hm

namespace hm {
struct BlkTab {                     // byte-chunk rank tables of the s = 1/2 block path
    void *dev = nullptr;
    int bytes = 0, oU = 0, oR0 = 0, oC = 0;
    uint16_t *lw = nullptr;         // K-bit words by popcount, each run in increasing order
    int lwoff[18] = {};             // run of popcount k starts at lw + lwoff[k]
};
}  // namespace hm

namespace hm {
constexpr int S1_KMAX = 10;         // s = 1 block path: at most 10 low sites (rank table of 4^K entries)
struct S1Tab {                      // tables of the s = 1 block path (s1blk.cu), one split K
    void *dev = nullptr;            // one device allocation holding the arrays below
    uint16_t *lut = nullptr;        // rank of every packed low word among words of its digit sum
    uint32_t *lw = nullptr;         // low words by digit sum, each run in rank order
    uint4 *blocks = nullptr;        // {h, off, k, rows} per block, in row order
    uint32_t *rl = nullptr;         // exchange rank tables of the low words (s1_sweep.cuh)
    uint32_t *rx = nullptr;
    int nlw = 0;
    int nblocks = 0, max_block = 0, K = -1;
    int lwoff[2 * S1_KMAX + 2] = {};
};
}  // namespace hm

struct hm_basis {
    hm::SectorView view;
    std::vector<uint64_t> D;        // host D(k, a), (N+1) x (S2*N+1)
    std::vector<uint64_t> cd;       // host CD, cd_len entries
    void *d_cd = nullptr;           // device copy (owned)
    void *d_scratch = nullptr;      // 256 bytes of device scratch (owned), e.g. exponents
    std::map<int, hm::BlkTab> blk_tabs;   // per split position K (owned device memory)
    std::map<std::string, void *> blk_ttabs;   // per-class target tables by layout (owned device memory)
    std::map<int, hm::S1Tab> s1_tabs;     // s = 1 block path, per split K (owned device memory)
    int parity = 0;                 // spin-flip basis (basis_build_flip): +1 / -1, view.dim halved
    int device = 0;
    // momentum basis (basis_build_momentum, momentum.cu): k = 0 or N/2, else -1.  view.dim is
    // then the number of representatives; mom_sector keeps the sector's own view
    int mom_k = -1;
    hm::SectorView mom_sector{};
    void *d_mom = nullptr;          // one allocation (owned): the sector map, then the list of representatives
    void *d_mom_map = nullptr;      // uint64 per sector index: representative | shift << 32 | period << 40
    void *d_mom_reps = nullptr;     // uint32 per representative: its sector index
};

namespace hm {

int digit_bits(int two_s);
// bonds of a momentum basis must map onto themselves under u -> u + 1 (momentum.cu)
int mom_check_bonds(const hm_basis *b, int n_bonds, const int32_t *u, const int32_t *v, const double *J);
// host helpers shared by the translation units
int build_tables(int n_sites, int two_s, int two_m, hm_basis *b);
int check_sector(int n_sites, int two_s, int two_m, int *A);

// ---------------------------------------------------------------------------------------
// bonds, normalised to p < q, passed to kernels by value
// ---------------------------------------------------------------------------------------
struct BondParams {
    int nb;
    int S2;
    unsigned char p[HM_MAX_BONDS], q[HM_MAX_BONDS];
    double jm[HM_MAX_BONDS];        // -J_b
    float jmf[HM_MAX_BONDS];        // -J_b rounded to float (FP32 paths)
    // exchange factors 1/2 sqrt(radicand product), indexed [a_p * 8 + a_q]:
    //   pdn: s+_p s-_q (a_p -> a_p - 1, a_q -> a_q + 1), radicand a_p(2s-a_p+1)(2s-a_q)(a_q+1)
    //   pup: s-_p s+_q (a_p -> a_p + 1, a_q -> a_q - 1), radicand (2s-a_p)(a_p+1)a_q(2s-a_q+1)
    double hs_pdn[64], hs_pup[64];
};

int make_bonds(const hm_basis *b, int n_bonds, const int32_t *u, const int32_t *v,
               const double *J, BondParams *out);
// y = H x on a momentum basis (momentum.cu), one vector
int mom_matvec(const hm_basis *b, const BondParams &bp, const void *x, void *y, int dtype, cudaStream_t st);
// terms of that product (1 per row + the exchanges that land on a basis state), into *nnz (device)
int mom_count_nnz(const hm_basis *b, const BondParams &bp, int64_t *nnz, cudaStream_t st);

// ---------------------------------------------------------------------------------------
// device codec
// ---------------------------------------------------------------------------------------
#ifdef __CUDA_ARCH__
#define HM_POPC64(x) __popcll(x)
#else
#define HM_POPC64(x) __builtin_popcountll(x)
#endif

__host__ __device__ __forceinline__ int dig(uint64_t w, int p, int bits) {
    return (int)((w >> (p * bits)) & ((1u << bits) - 1u));
}

// sum of the digits at positions < p
__host__ __device__ __forceinline__ int prefix_sum_below(uint64_t w, int p, int bits) {
    uint64_t m = (p * bits >= 64) ? ~0ull : ((1ull << (p * bits)) - 1ull);
    uint64_t x = w & m;
    if (bits == 1) return HM_POPC64(x);
    if (bits == 2) {
        x = (x & 0x3333333333333333ull) + ((x >> 2) & 0x3333333333333333ull);
        x = (x + (x >> 4)) & 0x0F0F0F0F0F0F0F0Full;
        return (int)((x * 0x0101010101010101ull) >> 56);
    }
    // bits == 4: byte sums fit (<= 30), total <= 16*15 = 240 fits a byte
    x = (x & 0x0F0F0F0F0F0F0F0Full) + ((x >> 4) & 0x0F0F0F0F0F0F0F0Full);
    return (int)((x * 0x0101010101010101ull) >> 56);
}

template <class I>
struct Codec {
    const I *cd;   // shared or global copy of CD
    int N, S2, A, bits, cd_w, cd_rowlen;

    __host__ __device__ __forceinline__ I at(int p, int S, int a) const {
        return cd[p * cd_rowlen + S * cd_w + a];
    }

    // Sec. 3.1: index -> packed digits
    __host__ __device__ __forceinline__ uint64_t decode(I i) const {
        uint64_t w = 0;
        int S = A;
        I r = i;
        for (int p = N - 1; p >= 1; --p) {
            const I *row = cd + p * cd_rowlen + S * cd_w;
            int amax = S < S2 ? S : S2;
            int a = 0;
            while (a < amax && row[a + 1] <= r) ++a;
            r -= row[a];
            S -= a;
            w |= (uint64_t)a << (p * bits);
        }
        return w | (uint64_t)S;
    }

    // Sec. 3.2: packed digits -> index
    __host__ __device__ __forceinline__ I encode(uint64_t w) const {
        int S = dig(w, 0, bits);
        I r = 0;
        for (int p = 1; p < N; ++p) {
            int a = dig(w, p, bits);
            S += a;
            r += at(p, S, a);
        }
        return r;
    }

    // index change when the digit at p moves by dp (+1/-1) and the digit at q > p by -dp:
    // only the rank terms of positions p..q change (prefix sums between them shift by dp)
    __host__ __device__ __forceinline__ I delta(uint64_t w, int p, int q, int dp) const {
        int S = prefix_sum_below(w, p, bits);
        I d = 0;
        for (int r = p; r <= q; ++r) {
            int a = dig(w, r, bits);
            S += a;
            int a2 = a + (r == p ? dp : (r == q ? -dp : 0));
            int S2n = S + (r < q ? dp : 0);
            d += at(r, S2n, a2) - at(r, S, a);
        }
        return d;
    }
};

// ---------------------------------------------------------------------------------------
// SplitMix64 (Steele, Lea, Flood, OOPSLA 2014): output t of the generator seeded with s
// is mix(s + (t+1) * 0x9E3779B97F4A7C15).
// ---------------------------------------------------------------------------------------
__host__ __device__ __forceinline__ uint64_t sm64(uint64_t seed, uint64_t t) {
    uint64_t z = seed + (t + 1ull) * 0x9E3779B97F4A7C15ull;
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
    return z ^ (z >> 31);
}

// number of blocks used by grid-stride kernels: fixed per device so reductions are
// reproducible run to run
// Raises (never lowers) the dynamic shared-memory limit of a kernel.  Several plans with
// different block sizes share one kernel, and launches captured into one graph after all of
// them were planned must each still fit.
template <class F>
inline cudaError_t raise_smem_limit(F kern, size_t bytes) {
    cudaFuncAttributes a;
    cudaError_t e = cudaFuncGetAttributes(&a, (const void *)kern);
    if (e != cudaSuccess) return e;
    if ((size_t)a.maxDynamicSharedSizeBytes >= bytes) return cudaSuccess;
    return cudaFuncSetAttribute((const void *)kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)bytes);
}
int grid_blocks(uint64_t rows, int threads);
int sm_count();

cudaStream_t as_stream(void *s);

}  // namespace hm
