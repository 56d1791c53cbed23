// blk.cuh -- block-structured row kernel for s = 1/2 sectors (shared by the matvec API,
// the Lanczos step and the batched finite-temperature driver).
//
// The sector states of N spins s = 1/2 with A flipped spins are the N-bit words of
// popcount A in increasing numerical order (Sec. 3: position N most significant).  Split
// a word into its high part h (positions K..N-1) and its low part l (positions 0..K-1).
// The rank of Sec. 3.2 is additive over positions, so
//     index(h, l) = off(h) + rank_K(l),   off(h) = sum over the ones of h of C(t, cnt),
// and all states with the same h form one contiguous block of C(K, A - popc(h)) rows.
// The kernel processes one block per CTA iteration:
//   * off(h) and the offsets of the blocks one exchange away are encoded once per block
//     with the paper's rank formula (D(p, c) = C(p, c) for s = 1/2);
//   * the low part is decoded and re-encoded with byte-chunk rank tables -- the same
//     rank sums of Sec. 3.2 precomputed 8 positions at a time:
//         rank_K(l) = U[popc(l)][l >> 8] + R0[l & 255];
//   * the block's own x values are staged in shared memory, so exchanges among the low
//     positions gather from shared memory; exchanges among the high positions move a
//     whole block to another block at a constant offset (coalesced gathers); exchanges
//     across the split touch one bit on each side.
// Couplings are grouped into classes of equal J (at most HM_BLK_MAXC).  In FP64 the
// hop sums of a class are exact int64 fixed-point sums (ef64.cuh), combined per row
// in double-float arithmetic: no FP64 instruction runs per row.
#pragma once

#include "ef64.cuh"
#include "hm_internal.cuh"

namespace hm {

constexpr int HM_BLK_MAXC = 4;      // coupling classes on the fast path
constexpr int HM_BLK_MAXG = 48;     // low bond groups
constexpr int HM_BLK_MAXB = 64;     // high / cross bonds

struct BlkParams {
    int N, K, H, A, nb1;            // nb1 = 2^(K-8)
    uint32_t dim;
    int max_block;
    int nc;
    float g_hi[HM_BLK_MAXC], g_lo[HM_BLK_MAXC];   // FP64 mode: -J_c / 4 as double-float
    float gq[HM_BLK_MAXC];                        // FP32 mode: -J_c / 4
    int ntot[HM_BLK_MAXC];                        // bonds in class c
    // low bonds grouped by (class, distance d, byte type): mask of start positions p;
    // type 0: both ends in byte 0, 1: both in byte 1, 2: across the bytes
    int nlg, lg_start[HM_BLK_MAXC + 1];
    uint32_t lg_mask[HM_BLK_MAXG];
    uint8_t lg_d[HM_BLK_MAXG], lg_type[HM_BLK_MAXG];
    // high bonds (positions relative to K) and cross bonds (p < K <= q), by class
    int nhb, hb_start[HM_BLK_MAXC + 1];
    uint8_t hb_p[HM_BLK_MAXB], hb_q[HM_BLK_MAXB];
    int ncb, cb_start[HM_BLK_MAXC + 1];
    uint8_t cb_p[HM_BLK_MAXB], cb_q[HM_BLK_MAXB];
    // device tables: U[(K+1) x nb1] (uint16), R0[256] (uint8), Cb[(N+1) x (A+1)] (uint32)
    const void *tab;
    int tab_bytes, off_U, off_R0, off_C;
};

// host: builds the plan; returns 0 if the bond list and sector take the fast path
int blk_plan(hm_basis *b, const BondParams &bp, int K, BlkParams *out);
size_t blk_smem_bytes(const BlkParams &P, int stage_bytes_per_row, int nvec);

// ---- device helpers ----------------------------------------------------------------------
struct BlkTabs {
    const uint16_t *U;
    const uint8_t *R0;
    const uint32_t *C;   // C[p * (A+1) + c] = D(p, c) = binomial(p, c), c <= A
};

__device__ __forceinline__ BlkTabs stage_blk_tables(const BlkParams &P, unsigned char *smem) {
    const uint32_t *src = (const uint32_t *)P.tab;
    uint32_t *dst = (uint32_t *)smem;
    for (int k = threadIdx.x; k < P.tab_bytes / 4; k += blockDim.x) dst[k] = src[k];
    BlkTabs t;
    t.U = (const uint16_t *)(smem + P.off_U);
    t.R0 = (const uint8_t *)(smem + P.off_R0);
    t.C = (const uint32_t *)(smem + P.off_C);
    return t;
}

// off(h): rank contribution of the high positions (Sec. 3.2) for a block whose low part
// holds k ones
__device__ __forceinline__ uint32_t blk_off(const BlkParams &P, const BlkTabs &T, uint32_t h, int k) {
    uint32_t off = 0;
    int cnt = k;
    uint32_t m = h;
    while (m) {
        const int t = __ffs(m) - 1;
        m &= m - 1;
        ++cnt;
        off += T.C[(P.K + t) * (P.A + 1) + cnt];
    }
    return off;
}

__device__ __forceinline__ uint32_t rank_low(const BlkParams &P, const BlkTabs &T, uint32_t l, int k) {
    return (uint32_t)T.U[k * P.nb1 + (l >> 8)] + (uint32_t)T.R0[l & 255u];
}

}  // namespace hm
