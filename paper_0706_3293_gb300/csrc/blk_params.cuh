// blk_params.cuh -- parameters of the s = 1/2 block path and the block offset off(h)
// (see blk.cuh for the layout); compiles under nvcc and NVRTC alike.
#pragma once

#include "hm_dev.cuh"

namespace hm {

constexpr int HM_BLK_MAXC = 4;      // coupling classes on the fast path
constexpr int HM_BLK_MAXG = 48;     // low bond groups
constexpr int HM_BLK_MAXB = 64;     // high / cross bonds
constexpr int HM_BLK_SL = 16;       // low-bond slots per class and byte type
constexpr int HM_BLK_SG = 6;        // exchange-count groups per class
constexpr int HM_BLK_SX = 8;        // cross-bond slots per class and byte

struct BlkParams {
    int N, K, H, A, nb1;            // nb1 = 2^(K-8)
    uint32_t dim;
    int max_block;
    int nc;
    float g_hi[HM_BLK_MAXC], g_lo[HM_BLK_MAXC];   // FP64 mode: -J_c / 4 as double-float
    float gq[HM_BLK_MAXC];                        // FP32 mode: -J_c / 4
    int ntot[HM_BLK_MAXC];                        // bonds in class c
    // integer-ratio classes: -J_c / 4 = Kc[c] * g0 exactly (small integers), so the row
    // value is g0 * sum_c Kc T_c, one exact integer; g0 = +-2^g0_exp when g0_pow2
    int iratio, g0_pow2, g0_exp;
    int Kc[HM_BLK_MAXC];
    double g0;
    float g0_hi, g0_lo;
    // low bonds grouped by (class, byte type, distance d): mask of start positions p;
    // type 0: both ends in byte 0, 1: both in byte 1, 2: across the bytes.  Groups of
    // class c and type t are [lg_cs[3c+t], lg_cs[3c+t+1]).
    int nlg, lg_cs[3 * HM_BLK_MAXC + 1];
    uint32_t lg_mask[HM_BLK_MAXG];
    uint8_t lg_d[HM_BLK_MAXG];
    // high bonds (positions relative to K) and cross bonds (p < K <= q), by class
    int nhb, hb_start[HM_BLK_MAXC + 1];
    uint8_t hb_p[HM_BLK_MAXB], hb_q[HM_BLK_MAXB];
    int ncb, cb_start[HM_BLK_MAXC + 1];
    uint8_t cb_p[HM_BLK_MAXB], cb_q[HM_BLK_MAXB];
    // device tables: U[(K+1) x nb1] (uint16), R0[256] (uint8), Cb[(N+1) x (A+1)] (uint32)
    const void *tab;
    int tab_bytes, off_U, off_R0, off_C;

    // ---- thread-per-row kernels (blk.cu): every bond a compile-time slot -------------
    // Low bonds by class c and byte type t (0: both ends in byte 0, 1: both in byte 1,
    // 2: across); slot s holds the distance d = q - p, the test bit 1 << p and the xor
    // masks that the exchange applies to the byte offsets 4 b0 and 4 b1 of the table
    // lookups below.  Cross bonds by class and the byte of their low end.
    int rows_ok;                                  // all bonds fit the slots below
    int kshift;                                   // K - 6: byte offset of row k of US is k << kshift
    int ln[HM_BLK_MAXC][3];
    uint8_t ld[HM_BLK_MAXC][3][HM_BLK_SL];
    uint32_t lvm[HM_BLK_MAXC][3][HM_BLK_SL];
    uint16_t lxa[HM_BLK_MAXC][3][HM_BLK_SL], lxb[HM_BLK_MAXC][3][HM_BLK_SL];
    // exchange counts of the low bonds: sum over groups g of popc((l ^ l >> gd) & gm)
    int lgn[HM_BLK_MAXC];
    uint8_t lgd[HM_BLK_MAXC][HM_BLK_SG];
    uint32_t lgm[HM_BLK_MAXC][HM_BLK_SG];
    int xn[HM_BLK_MAXC][2];
    uint16_t xxa[HM_BLK_MAXC][2][HM_BLK_SX];      // 4 << p (byte 0) or 4 << (p - 8) (byte 1)
    // the same cross bonds in one list for the per-block setup: low end p, high end
    // q - K, slot index (2 c + t) * HM_BLK_SX + s
    int nxf;
    uint8_t xf_p[HM_BLK_MAXB], xf_q[HM_BLK_MAXB], xf_dst[HM_BLK_MAXB];
    const uint16_t *lw;                           // low words by popcount (BlkTab::lw)
    int lwoff[18];
    // spin-flip basis (M = 0): parity +1 / -1 of the representatives' vectors, 0 otherwise;
    // the blocks swept are those whose site N-1 (high bit H - 1) is up
    int par;
    // per-bond couplings (more than HM_BLK_MAXC distinct J): every bond sits in the slots of
    // class 0 and a row is y_i = g0 x_i + sum over its allowed exchanges of
    // h_b (x_i - x_target), h_b = J_b / 2, g0 = -sum_b J_b / 4 (Eq. E-2-1).  In FP64 the
    // coefficients are integers scaled by 2^pb_s (|C| < 2^62): C_b = round(h_b 2^pb_s),
    // pb_c0 = round(g0 2^pb_s), and a row is one exact int128 sum, rounded once
    int perbond;
    int pb_s;
    long long pb_c0;
    double pb_g0;
    uint8_t pb_lb[3][HM_BLK_SL], pb_xb[2][HM_BLK_SX];   // bond index of each low / cross slot
    uint8_t pb_hbb[HM_BLK_MAXB];                      // bond index of each high bond
    long long pb_hc[HM_BLK_MAXB];                     // C_b of each high bond (hb_p / hb_q order)
    // bond-correlation plan (one chunk of bonds, per-bond slots): the block setup keeps the
    // high targets uncompacted, hbi[j] for high bond j or ~0 when its spins are parallel
    int bcmode;
    // per-class target tables (row policy "table", jit.cu): the row of rank r in the low-word
    // list of class k (list position g = lwoff[k] + r) has tt_n 16-bit entries, eight to a
    // 16-byte chunk, entry s in chunk s / 8 at tt[(s / 8) * tt_stride + g]: first the byte
    // offsets of the low slots' target rows in the staged block (the zero row when the two
    // spins are parallel), then for each low end p of a cross bond the byte offset of the rank
    // of l ^ 2^p among the words of its popcount
    const uint4 *tt;
    uint32_t tt_stride;
    int tt_n, tt_ncross, tt_cross_p[8];
    // the low slots as edge-disjoint triangles of bonds (a, b), (b, c), (a, c), whose spin
    // pairs hold exactly zero or two unequal pairs, so two gathers (two entries) serve three
    // slots, then single slots.  The first gathered edge of a triangle is always class
    // tri_ca; the second is (b, c), class tri_ca, when the spins of a and c are parallel,
    // else (a, c), class tri_cb: tri_a and tri_c are the sites of (a, c)
    int tt_ntri, tt_nsgl;
    uint8_t tt_tri_ca[16], tt_tri_cb[16], tt_tri_a[16], tt_tri_c[16], tt_sgl_c[48];
    // two-pass FP64 Lanczos product (integer-ratio classes): pass 1 applies the near bonds
    // and stores each row's exact integer class sum, pass 2 adds the far bonds (those
    // reaching the top sites) and rounds once.  rot: pass 2 takes the blocks in the order of
    // the high word rotated so that its top rot bits vary fastest
    int split, rot;
};


struct BlkTabs {
    const uint16_t *U;
    const uint8_t *R0;
    const uint32_t *C;   // C[p * (A+1) + c] = D(p, c) = binomial(p, c), c <= A
};

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

}  // namespace hm
