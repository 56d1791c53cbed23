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

#include <climits>

#include "blk_params.cuh"
#include "ef64.cuh"
#include "hm_internal.cuh"

namespace hm {

// host: builds the plan; returns 0 if the bond list and sector take the fast path.  use:
// bit t set = bond t is applied (a pass of the two-pass product applies a subset; the
// coupling classes always come from the whole list, so both passes share them)
int blk_plan(hm_basis *b, const BondParams &bp, int K, BlkParams *out, bool bond_corr = false,
             uint64_t use = ~0ull);

// ---- device helpers ----------------------------------------------------------------------
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

__device__ __forceinline__ uint32_t rank_low(const BlkParams &P, const BlkTabs &T, uint32_t l, int k) {
    return (uint32_t)T.U[k * P.nb1 + (l >> 8)] + (uint32_t)T.R0[l & 255u];
}

}  // namespace hm

namespace hm {

// ---- per-block setup shared by the block kernels -------------------------------------------
// Shared scratch of one block: compacted high-exchange offsets per class, cross-exchange
// targets.
struct BlkShared {
    int *hcd;             // [HM_BLK_MAXB] offsets (target row - own row) of the valid high exchanges
    int *hcs;             // [HM_BLK_MAXC + 1] class c owns hcd[hcs[c] .. hcs[c+1])
    uint32_t *coff;       // [HM_BLK_MAXB] sector offset of the cross target block
    int8_t *ck;           // [HM_BLK_MAXB] low popcount of the cross target (-1: none)
    uint8_t *cbq;         // [HM_BLK_MAXB] bit q of h for the cross bond
};

__host__ __device__ __forceinline__ size_t blk_al16(size_t x) { return (x + 15) & ~(size_t)15; }

// bytes of BlkShared after the staged rows
__host__ __device__ __forceinline__ size_t blk_shared_bytes(int max_block) {
    (void)max_block;
    return blk_al16(HM_BLK_MAXB * 4) + blk_al16((HM_BLK_MAXC + 1) * 4) + blk_al16(HM_BLK_MAXB * 4) +
           blk_al16(HM_BLK_MAXB) * 2;
}

__device__ __forceinline__ BlkShared blk_carve(unsigned char *p, int max_block) {
    BlkShared s;
    (void)max_block;
    s.hcd = (int *)p; p += blk_al16(HM_BLK_MAXB * 4);
    s.hcs = (int *)p; p += blk_al16((HM_BLK_MAXC + 1) * 4);
    s.coff = (uint32_t *)p; p += blk_al16(HM_BLK_MAXB * 4);
    s.ck = (int8_t *)p; p += blk_al16(HM_BLK_MAXB);
    s.cbq = (uint8_t *)p;
    return s;
}

// Offsets of the block one exchange away (high and cross bonds), for the block of high
// word h whose low part holds k ones (its low words, in rank order, are the run of
// popcount k of BlkParams::lw).  Warp 0 lists the valid high exchanges (two bonds a lane,
// compacted by class through its ballots), warp 1 the cross exchanges; no barrier here:
// the caller syncs before reading sh.  Returns the block's row count; *off_out = off(h).
__device__ __forceinline__ int blk_setup_block(const BlkParams &P, const BlkTabs &tb, uint32_t h, int k,
                                               const BlkShared &sh, uint32_t *off_out) {
    const uint32_t off = blk_off(P, tb, h, k);
    const int n = (int)tb.C[P.K * (P.A + 1) + k];
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    if (warp == 0) {
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
        if (lane <= HM_BLK_MAXC) {                 // class c starts at the valid ones before hb_start[c]
            const int e = P.hb_start[lane];
            sh.hcs[lane] = e >= 32 ? __popc(b0) + __popc(e >= 64 ? b1 : b1 & ((1u << (e - 32)) - 1u))
                                   : __popc(b0 & ((1u << e) - 1u));
        }
    } else if (warp == 1) {
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
    *off_out = off;
    return n;
}

// f(r2) for every allowed exchange of class c among the low positions (targets in the
// same block); returns their number
template <class F>
__device__ __forceinline__ int blk_low_hops(const BlkParams &P, const BlkTabs &tb, int c, uint32_t l,
                                            uint32_t r, const uint16_t *Uk, F &&f) {
    const uint32_t R0own = tb.R0[l & 255u];
    const uint32_t R1own = r - R0own;
    int mc = 0;
    for (int g = P.lg_cs[3 * c]; g < P.lg_cs[3 * c + 1]; ++g) {        // inside byte 0
        const int d = P.lg_d[g];
        const uint32_t pat = 1u | (1u << d);
        uint32_t m = ((l >> d) ^ l) & P.lg_mask[g];
        while (m) {
            const int p = __ffs(m) - 1;
            m &= m - 1;
            f(R1own + tb.R0[(l ^ (pat << p)) & 255u]);
            ++mc;
        }
    }
    for (int g = P.lg_cs[3 * c + 1]; g < P.lg_cs[3 * c + 2]; ++g) {    // inside byte 1
        const int d = P.lg_d[g];
        const uint32_t pat = 1u | (1u << d);
        uint32_t m = ((l >> d) ^ l) & P.lg_mask[g];
        while (m) {
            const int p = __ffs(m) - 1;
            m &= m - 1;
            f(R0own + Uk[(l ^ (pat << p)) >> 8]);
            ++mc;
        }
    }
    for (int g = P.lg_cs[3 * c + 2]; g < P.lg_cs[3 * c + 3]; ++g) {    // across the bytes
        const int d = P.lg_d[g];
        const uint32_t pat = 1u | (1u << d);
        uint32_t m = ((l >> d) ^ l) & P.lg_mask[g];
        while (m) {
            const int p = __ffs(m) - 1;
            m &= m - 1;
            const uint32_t l2 = l ^ (pat << p);
            f((uint32_t)Uk[l2 >> 8] + tb.R0[l2 & 255u]);
            ++mc;
        }
    }
    return mc;
}

// f(j) (j: row inside the sector) for every allowed exchange of class c across the split
template <class F>
__device__ __forceinline__ int blk_cross_hops(const BlkParams &P, const BlkTabs &tb, int c, uint32_t l,
                                              const BlkShared &sh, F &&f) {
    int mc = 0;
    for (int e = P.cb_start[c]; e < P.cb_start[c + 1]; ++e) {
        const int p = P.cb_p[e];
        if ((((l >> p) & 1u) != sh.cbq[e]) && sh.ck[e] >= 0) {
            const uint32_t l2 = l ^ (1u << p);
            f(sh.coff[e] + rank_low(P, tb, l2, sh.ck[e]));
            ++mc;
        }
    }
    return mc;
}

}  // namespace hm
