// s1blk.cuh -- plan and host entry points of the s = 1 block-structured products (s1blk.cu).
#pragma once

#include "hm_internal.cuh"

namespace hm {

constexpr int S1_NT = 512;
constexpr int S1_MAXB = 96;          // bonds of each kind

struct S1Plan {
    int N, K, H, A, nblocks, max_block;
    const uint16_t *lut;             // [4^K]: rank_K of each packed low word among words of its digit sum
    const uint32_t *lw;              // packed low words by digit sum k, each run in rank order
    const uint4 *blocks;             // per block, in row order: {h, off, k, rows}
    const uint32_t *cd;              // the sector's CD table (cd_w, cd_rowlen as in SectorView)
    int cd_w, cd_rowlen, cd_len;
    int lwoff[2 * S1_KMAX + 2];      // digit sum k owns lw[lwoff[k] .. lwoff[k + 1])
    int nlo, nhi, ncr;
    uint8_t lo_p[S1_MAXB], lo_q[S1_MAXB];   // both ends below K
    uint8_t hi_p[S1_MAXB], hi_q[S1_MAXB];   // both ends at K or above (relative to K)
    uint8_t cr_p[S1_MAXB], cr_q[S1_MAXB];   // low end p, high end q (relative to K)
    float lo_j[S1_MAXB], hi_j[S1_MAXB], cr_j[S1_MAXB];   // -J_b
};

// plan of the s = 1 block path for these bonds; 1 when it does not apply (the caller runs
// the general row kernel), < 0 on error.  Builds the basis's tables on first use.
int s1_plan(hm_basis *b, const BondParams &bp, S1Plan *P);
// y = H x, FP32, one vector
int s1_matvec(const S1Plan &P, const float *x, float *y, cudaStream_t st);
// Lanczos product, FP32: q_prev <- sigma H q - gamma q_prev; part[block] = (sigma q . u)
int s1_lz32(const S1Plan &P, const float *qc, float *qp, const LzScalars *S, double *part, cudaStream_t st);
// number of blocks of a basis's s = 1 path with K = min(10, N - 2) (0 when it does not apply)
uint64_t s1_block_count(const hm_basis *b);

}  // namespace hm
