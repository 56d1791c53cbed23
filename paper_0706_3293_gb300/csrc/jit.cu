// jit.cu -- the s = 1/2 Lanczos products specialised to one bond list at run time.
//
// The generic block kernels (blk.cu) read every bond slot from the kernel parameters and
// enter the runs of slots through switches.  Here the slots of a plan are written out as
// straight-line code with their positions and masks as literals, the in-byte exchanges
// go through delta tables (gen_row), the result is compiled for sm_103a with NVRTC and
// loaded with cudaLibraryLoadData.  Both variants run the same bodies (blk_sweep.cuh);
// in FP64 both form the same exact integer sums, so their outputs agree bit for bit.
// The generic kernel stays the fallback when NVRTC is not available (HM_JIT=0 selects
// it on purpose).  Two row policies: the slots written out (default), or per-byte delta
// tables (HM_JIT_ROW=delta: fewer instructions and shared-memory wavefronts, faster where
// the hop gathers hit L2, as for N = 28; slower at N = 32).  HM_JIT_CTAS=2 trades the
// third resident CTA per SM for 64 registers a thread.
#include <dlfcn.h>
#include <nvrtc.h>

#include <cstdarg>
#include <cstdio>
#include <cstdlib>
#include <algorithm>
#include <cstring>
#include <map>
#include <mutex>
#include <set>
#include <string>
#include <vector>

#include "blk.cuh"
#include "blk_sweep.cuh"
#include "s1blk.cuh"
#include "jit_embed.inc"   // kJitHeaderNames / kJitHeaderTexts: the .cuh files above, as text

#ifndef HM_CUDA_LIBDIR
#define HM_CUDA_LIBDIR "/usr/local/cuda/lib64"
#endif

namespace hm {
long long pb_coef(const BlkParams &P, double h);   // blk.cu: round(h 2^pb_s)

namespace {

struct Nvrtc {
    bool tried = false, ok = false;
    std::string why;
    nvrtcResult (*create)(nvrtcProgram *, const char *, const char *, int, const char *const *,
                          const char *const *) = nullptr;
    nvrtcResult (*compile)(nvrtcProgram, int, const char *const *) = nullptr;
    nvrtcResult (*cubin_size)(nvrtcProgram, size_t *) = nullptr;
    nvrtcResult (*cubin)(nvrtcProgram, char *) = nullptr;
    nvrtcResult (*log_size)(nvrtcProgram, size_t *) = nullptr;
    nvrtcResult (*log)(nvrtcProgram, char *) = nullptr;
    nvrtcResult (*destroy)(nvrtcProgram *) = nullptr;
};

std::mutex g_mu;
Nvrtc g_nv;
std::map<std::string, const void *> g_cache;   // (device, source) -> kernel handle
std::map<const void *, int> g_pad;              // kernel handle -> pad elements after the staged rows
std::set<std::string> g_failed;

bool load_nvrtc() {
    if (g_nv.tried) return g_nv.ok;
    g_nv.tried = true;
    const char *names[] = {"libnvrtc.so.13", "libnvrtc.so", HM_CUDA_LIBDIR "/libnvrtc.so.13",
                           HM_CUDA_LIBDIR "/libnvrtc.so"};
    void *h = nullptr;
    for (const char *n : names)
        if ((h = dlopen(n, RTLD_NOW | RTLD_LOCAL)) != nullptr) break;
    if (!h) { g_nv.why = "libnvrtc not found"; return false; }
    auto sym = [&](const char *s) { return dlsym(h, s); };
    g_nv.create = (decltype(g_nv.create))sym("nvrtcCreateProgram");
    g_nv.compile = (decltype(g_nv.compile))sym("nvrtcCompileProgram");
    g_nv.cubin_size = (decltype(g_nv.cubin_size))sym("nvrtcGetCUBINSize");
    g_nv.cubin = (decltype(g_nv.cubin))sym("nvrtcGetCUBIN");
    g_nv.log_size = (decltype(g_nv.log_size))sym("nvrtcGetProgramLogSize");
    g_nv.log = (decltype(g_nv.log))sym("nvrtcGetProgramLog");
    g_nv.destroy = (decltype(g_nv.destroy))sym("nvrtcDestroyProgram");
    g_nv.ok = g_nv.create && g_nv.compile && g_nv.cubin_size && g_nv.cubin && g_nv.log_size && g_nv.log &&
              g_nv.destroy;
    if (!g_nv.ok) g_nv.why = "libnvrtc lacks an entry point";
    return g_nv.ok;
}

bool verbose() {
    const char *v = getenv("HM_JIT_VERBOSE");
    return v && v[0] == '1';
}

void put(std::string &s, const char *fmt, ...) __attribute__((format(printf, 2, 3)));
void put(std::string &s, const char *fmt, ...) {
    va_list ap, ap2;
    va_start(ap, fmt);
    va_copy(ap2, ap);
    const int n = vsnprintf(nullptr, 0, fmt, ap);
    va_end(ap);
    if (n > 0) {
        std::vector<char> buf((size_t)n + 1);
        vsnprintf(buf.data(), buf.size(), fmt, ap2);
        s.append(buf.data(), (size_t)n);
    }
    va_end(ap2);
}

// The row policy of a plan written out slot by slot: RowGeneric (blk_sweep.cuh) with
// every count, shift and mask a literal, in RowGeneric's order (each run from its last
// slot down, so FP32 sums round the same way).  A failed exchange reads byte-0 table
// entry 0 and a zero element past the staged rows instead of its own lookups: all such
// lanes hit the same words (broadcasts), and the add needs no select.
// the add of cross slot `dst`: a target in the complement block (spin-flip basis, bond
// on site N-1) lies below its base and carries the parity sign
const char *xadd(const BlkParams &P, int dst) {
    for (int e = 0; e < P.nxf; ++e)
        if (P.xf_dst[e] == dst && P.par && P.xf_q[e] == P.H - 1)
            return P.par < 0 ? "a -= gx(x_.base - v_)" : "a += gx(x_.base - v_)";
    return "a += gx(x_.base + v_)";
}

std::string gen_row_slots(const BlkParams &P) {
    std::string s;
    s += "struct RowJit {\n"
         "static constexpr int kPad = hm::BLK_XPAD;\n"
         "static constexpr bool kRelUS = false;\n"
         "static constexpr bool kPerBond = false;\n"
         "static constexpr bool kBC = false;\n"
         "template <class Sv>\n"
         "static __device__ __forceinline__ void stage(const hm::BlkParams &P, unsigned char *dyn) {\n"
         "    hm::RowGeneric<1>::stage<Sv>(P, dyn);\n"
         "    if (threadIdx.x == 0) *(Sv *)(dyn + (P.max_block + hm::BLK_XPAD - 1) * sizeof(Sv)) = Sv(0);\n"
         "}\n"
         "template <class Sv>\n"
         "static __device__ __forceinline__ void block(const hm::BlkParams &, uint32_t) {}\n"
         "template <class Sv, class G>\n"
         "static __device__ __forceinline__ void sums(const hm::BlkParams &P, const hm::BlkMeta &B,\n"
         "        const unsigned char *Xsb, const unsigned char *Xg, uint32_t l, uint32_t r, const G &gx, Sv xo,\n"
         "        Sv *acc, int *cnt) {\n"
         "    const uint32_t l4 = l << 2, lh4 = (l >> 8) << 2, lh4k = lh4 | B.kofs;\n"
         "    const uint32_t R0own = hm::r0s_at(l4 & 0x3FCu), R1own = hm::us_at(lh4k);\n"
         "    const uint32_t zo = (uint32_t)((P.max_block + hm::BLK_XPAD - 1) * sizeof(Sv));   // zero slot\n"
         "    (void)R0own; (void)R1own; (void)lh4; (void)gx; (void)xo; (void)zo;\n";
    // the distances that occur among the low bonds and count groups
    std::set<int> ds;
    for (int c = 0; c < P.nc; ++c) {
        for (int t = 0; t < 3; ++t)
            for (int k = 0; k < P.ln[c][t]; ++k) ds.insert(P.ld[c][t][k]);
        for (int g = 0; g < P.lgn[c]; ++g) ds.insert(P.lgd[c][g]);
    }
    for (int d : ds) put(s, "    const uint32_t z%d = l ^ (l >> %d);\n", d, d);
    for (int c = 0; c < P.nc; ++c) {
        put(s, "    {   // class %d\n        Sv a = Sv(0);\n        int m = 0;\n", c);
        for (int k = P.ln[c][0] - 1; k >= 0; --k)
            put(s, "        { const bool t = (z%d & 0x%xu) != 0u; const uint32_t o = R1own + hm::r0s_at(t ? (l4 ^ 0x%xu) & 0x3FCu : 0u); "
                   "a += *(const Sv *)(Xsb + (t ? o : zo)); }\n",
                P.ld[c][0][k], P.lvm[c][0][k], (unsigned)P.lxa[c][0][k]);
        for (int k = P.ln[c][1] - 1; k >= 0; --k)
            put(s, "        { const bool t = (z%d & 0x%xu) != 0u; const uint32_t o = R0own + hm::us_at(lh4k ^ 0x%xu); "
                   "a += *(const Sv *)(Xsb + (t ? o : zo)); }\n",
                P.ld[c][1][k], P.lvm[c][1][k], (unsigned)P.lxb[c][1][k]);
        for (int k = P.ln[c][2] - 1; k >= 0; --k)
            put(s, "        { const bool t = (z%d & 0x%xu) != 0u; const uint32_t o = hm::us_at(lh4k ^ 0x%xu) + "
                   "hm::r0s_at(t ? (l4 ^ 0x%xu) & 0x3FCu : 0u); a += *(const Sv *)(Xsb + (t ? o : zo)); }\n",
                P.ld[c][2][k], P.lvm[c][2][k], (unsigned)P.lxb[c][2][k], (unsigned)P.lxa[c][2][k]);
        for (int g = P.lgn[c] - 1; g >= 0; --g) put(s, "        m += __popc(z%d & 0x%xu);\n", P.lgd[c][g], P.lgm[c][g]);
        for (int k = P.xn[c][0] - 1; k >= 0; --k)
            put(s, "        { const hm::XSlot x_ = B.xs[%d]; const uint32_t v_ = hm::us_at(lh4 | x_.kofs2) + "
                   "hm::r0s_at((l4 ^ 0x%xu) & 0x3FCu); if ((l ^ x_.wm) & x_.vm) { %s; ++m; } }\n",
                (2 * c) * HM_BLK_SX + k, (unsigned)P.xxa[c][0][k], xadd(P, (2 * c) * HM_BLK_SX + k));
        for (int k = P.xn[c][1] - 1; k >= 0; --k)
            put(s, "        { const hm::XSlot x_ = B.xs[%d]; const uint32_t v_ = hm::us_at((lh4 ^ 0x%xu) | x_.kofs2) + "
                   "R0own; if ((l ^ x_.wm) & x_.vm) { %s; ++m; } }\n",
                (2 * c + 1) * HM_BLK_SX + k, (unsigned)P.xxa[c][1][k], xadd(P, (2 * c + 1) * HM_BLK_SX + k));
        put(s, "        a += hm::blk_high_sum<Sv>(B, %d, Xg, r, gx);\n", c);
        if (P.par) {
            put(s, "        a %s= hm::blk_flip_sum<Sv>(B, %d, Xg, r, gx);\n", P.par < 0 ? "-" : "+", c);
            put(s, "        acc[%d] = a;\n        cnt[%d] = m + (B.he[%d] - B.hs[%d]) + (B.x->fe[%d] - B.x->fs[%d]);\n    }\n",
                c, c, c, c, c, c);
        } else {
            put(s, "        acc[%d] = a;\n        cnt[%d] = m + (B.he[%d] - B.hs[%d]);\n    }\n", c, c, c, c);
        }
    }
    s += "}\n};\n";
    return s;
}

// The row policy of a plan with per-class target tables (BlkParams::tt, blk.cu
// blk_target_table): the row's table entries are read as 16-byte chunks (consecutive rows
// read consecutive chunks, so the loads are coalesced and served from L2).  A triangle of
// low bonds is two shared-memory gathers at the byte offsets its two entries hold, added to
// its two classes as its code says; a single low slot is one gather (the zero row when the
// spins are parallel).  No rank-table reads and no per-slot spin test; the exchange counts
// come from the plan's count groups (popc of z_d & mask).  Cross and high exchanges as in
// gen_row_slots.
std::string gen_row_table(const BlkParams &P) {
    std::string s;
    s += "struct RowJit {\n"
         "static constexpr int kPad = hm::BLK_XPAD;\n"
         "static constexpr bool kRelUS = false;\n"
         "static constexpr bool kPerBond = false;\n"
         "static constexpr bool kBC = false;\n"
         "template <class Sv>\n"
         "static __device__ __forceinline__ void stage(const hm::BlkParams &P, unsigned char *dyn) {\n"
         "    if (threadIdx.x == 0) *(Sv *)(dyn + (P.max_block + hm::BLK_XPAD - 1) * sizeof(Sv)) = Sv(0);\n"
         "}\n"
         "template <class Sv>\n"
         "static __device__ __forceinline__ void block(const hm::BlkParams &, uint32_t) {}\n"
         "template <class Sv, class G>\n"
         "static __device__ __forceinline__ void sums(const hm::BlkParams &P, const hm::BlkMeta &B,\n"
         "        const unsigned char *Xsb, const unsigned char *Xg, uint32_t l, uint32_t r, const G &gx, Sv xo,\n"
         "        Sv *acc, int *cnt) {\n"
         "    (void)l; (void)gx; (void)xo; (void)Xg;\n"
         "    const uint4 *tt = P.tt + (B.lwo + r);\n";
    const int nch = (P.tt_n + 7) / 8;
    for (int j = 0; j < nch; ++j) put(s, "    const uint4 q%d = hm::ldg_v4(tt + %uu);\n", j, (unsigned)j * P.tt_stride);
    static const char *comp[4] = {"x", "y", "z", "w"};
    auto entry = [&](int e) {
        char buf[64];
        const int j = e / 8, c = (e % 8) / 2;
        if (e % 2 == 0) snprintf(buf, sizeof buf, "(q%d.%s & 0xFFFFu)", j, comp[c]);
        else snprintf(buf, sizeof buf, "(q%d.%s >> 16)", j, comp[c]);
        return std::string(buf);
    };
    const int ntri = P.tt_ntri, nsgl = P.tt_nsgl, ecross = 2 * ntri + nsgl;
    auto cross_entry = [&](int c, int t, int k) {
        const int p = __builtin_ctz((unsigned)P.xxa[c][t][k]) - 2 + (t == 1 ? 8 : 0);
        for (int i = 0; i < P.tt_ncross; ++i)
            if (P.tt_cross_p[i] == p) return ecross + i;
        return -1;
    };
    // the count groups' distances
    std::set<int> ds;
    for (int c = 0; c < P.nc; ++c)
        for (int g = 0; g < P.lgn[c]; ++g) ds.insert(P.lgd[c][g]);
    for (int d : ds) put(s, "    const uint32_t z%d = l ^ (l >> %d);\n", d, d);
    s += "#define XS(o) (*(const Sv *)(Xsb + (o)))\n";
    for (int c = 0; c < P.nc; ++c) {
        put(s, "    Sv a%d = Sv(0);\n    int m%d = 0;\n", c, c);
        for (int g = P.lgn[c] - 1; g >= 0; --g) put(s, "    m%d += __popc(z%d & 0x%xu);\n", c, P.lgd[c][g], P.lgm[c][g]);
    }
    for (int t = 0; t < ntri; ++t) {
        const int ca = P.tt_tri_ca[t], cb = P.tt_tri_cb[t];
        put(s, "    { const Sv x1 = XS(%s), x2 = XS(%s);\n", entry(2 * t).c_str(), entry(2 * t + 1).c_str());
        if (ca == cb) {
            put(s, "      a%d += x1 + x2; }\n", ca);
        } else {
            // the second gathered edge is (b, c), class ca, when the spins of a and c are
            // parallel, else (a, c), class cb
            const int a = P.tt_tri_a[t], c = P.tt_tri_c[t], d = c - a;
            if (ds.count(d)) put(s, "      const Sv x2a = ((z%d >> %d) & 1u) ? Sv(0) : x2;\n", d, a);
            else put(s, "      const Sv x2a = (((l >> %d) ^ (l >> %d)) & 1u) ? Sv(0) : x2;\n", a, c);
            put(s, "      a%d += x1 + x2a; a%d += x2 - x2a; }\n", ca, cb);
        }
    }
    for (int i = 0; i < nsgl; ++i) put(s, "    a%d += XS(%s);\n", P.tt_sgl_c[i], entry(2 * ntri + i).c_str());
    // cross exchanges; in a spin-flip basis those moving site N-1 up gather row n - 1 - r of the
    // complement block, below its base, with the parity sign
    for (int c = 0; c < P.nc; ++c)
        for (int t = 0; t < 2; ++t)
            for (int k = 0; k < P.xn[c][t]; ++k) {
                const int dst = (2 * c + t) * HM_BLK_SX + k;
                const char *add = "a%d += gx(x_.base + %s)";
                for (int e2 = 0; e2 < P.nxf; ++e2)
                    if (P.xf_dst[e2] == dst && P.par && P.xf_q[e2] == P.H - 1)
                        add = P.par < 0 ? "a%d -= gx(x_.base - %s)" : "a%d += gx(x_.base - %s)";
                char buf[160];
                snprintf(buf, sizeof buf, add, c, entry(cross_entry(c, t, k)).c_str());
                put(s, "    { const hm::XSlot x_ = B.xs[%d]; if ((l ^ x_.wm) & x_.vm) { %s; ++m%d; } }\n", dst, buf, c);
            }
    // high gathers in flight (HM_JIT_HIGH = 1, 2, 4): more hide more latency, fewer keep the
    // registers (and local-memory spills) down
    int nh = 4;
    if (const char *v = getenv("HM_JIT_HIGH")) nh = atoi(v) == 1 ? 1 : atoi(v) == 2 ? 2 : 4;
    // the last round predicated (blk_high_sum's PRED): FP32 rows and the FP64 rows of the
    // sector product; the FP64 spin-flip rows keep the tail loop
    for (int c = 0; c < P.nc; ++c) {
        if (P.par)
            put(s, "    acc[%d] = a%d + hm::blk_high_sum<Sv, %d>(B, %d, Xg, r, gx) %s hm::blk_flip_sum<Sv>(B, %d, Xg, r, gx);\n"
                   "    cnt[%d] = m%d + (B.he[%d] - B.hs[%d]) + (B.x->fe[%d] - B.x->fs[%d]);\n",
                c, c, nh, c, P.par < 0 ? "-" : "+", c, c, c, c, c, c, c);
        else
            put(s, "    acc[%d] = a%d + hm::blk_high_sum<Sv, %d, true>(B, %d, Xg, r, gx);\n    cnt[%d] = m%d + (B.he[%d] - B.hs[%d]);\n",
                c, c, nh, c, c, c, c, c);
    }
    s += "#undef XS\n}\n};\n";
    return s;
}

// The row policy of a per-bond plan (BlkParams::perbond): the slots of class 0 written out
// as in gen_row_slots, each with its own coefficient h_b = J_b / 2 as a literal, summed
// as h_b (x_i - x_t) (blk_sweep.cuh, per-bond rows).  A slot whose spins are parallel reads
// a fixed address (a broadcast) and adds a zero difference.
std::string gen_row_pb_table(const BlkParams &P, const BondParams &bp);

std::string gen_row_pb(const BlkParams &P, const BondParams &bp) {
    if (P.tt) return gen_row_pb_table(P, bp);
    auto hb = [&](int t) { return -bp.jm[t] / 2.0; };
    // coefficient arguments of hm::pb_mac: C_b (integer, FP64 rows) and h_b (float, FP32 rows)
    auto cf = [&](int t) {
        char buf[96];
        snprintf(buf, sizeof buf, "%lldLL, %.9gf", pb_coef(P, hb(t)), hb(t));
        return std::string(buf);
    };
    std::string s;
    s += "struct RowJit {\n"
         "static constexpr int kPad = hm::BLK_XPAD;\n"
         "static constexpr bool kRelUS = false;\n"
         "static constexpr bool kPerBond = true;\n"
         "static constexpr bool kBC = false;\n"
         "template <class Sv>\n"
         "static __device__ __forceinline__ void stage(const hm::BlkParams &P, unsigned char *dyn) {\n"
         "    hm::RowGeneric<1>::stage<Sv>(P, dyn);\n"
         "}\n"
         "template <class Sv>\n"
         "static __device__ __forceinline__ void block(const hm::BlkParams &, uint32_t) {}\n"
         "template <class Sv, class G>\n"
         "static __device__ __forceinline__ typename hm::PbAcc<Sv>::T sums_pb(const hm::BlkParams &P,\n"
         "        const hm::BlkMeta &B, const unsigned char *Xsb, const unsigned char *Xg, uint32_t l, uint32_t r,\n"
         "        const G &gx, Sv xo) {\n"
         "    const uint32_t l4 = l << 2, lh4 = (l >> 8) << 2, lh4k = lh4 | B.kofs;\n"
         "    const uint32_t R0own = hm::r0s_at(l4 & 0x3FCu), R1own = hm::us_at(lh4k);\n"
         "    const uint32_t zo = (uint32_t)((P.max_block + hm::BLK_XPAD - 1) * sizeof(Sv));   // fixed address\n"
         "    (void)R0own; (void)R1own; (void)lh4; (void)gx; (void)zo;\n"
         "    typename hm::PbAcc<Sv>::T a = 0;\n";
    std::set<int> ds;
    for (int t = 0; t < 3; ++t)
        for (int k = 0; k < P.ln[0][t]; ++k) ds.insert(P.ld[0][t][k]);
    for (int d : ds) put(s, "    const uint32_t z%d = l ^ (l >> %d);\n", d, d);
    for (int k = P.ln[0][0] - 1; k >= 0; --k)
        put(s, "    { const bool t = (z%d & 0x%xu) != 0u; const uint32_t o = R1own + hm::r0s_at(t ? (l4 ^ 0x%xu) & 0x3FCu : 0u); "
               "const Sv x = *(const Sv *)(Xsb + (t ? o : zo)); a = hm::pb_mac(%s, t ? xo - x : Sv(0), a); }\n",
            P.ld[0][0][k], P.lvm[0][0][k], (unsigned)P.lxa[0][0][k], cf(P.pb_lb[0][k]).c_str());
    for (int k = P.ln[0][1] - 1; k >= 0; --k)
        put(s, "    { const bool t = (z%d & 0x%xu) != 0u; const uint32_t o = R0own + hm::us_at(lh4k ^ 0x%xu); "
               "const Sv x = *(const Sv *)(Xsb + (t ? o : zo)); a = hm::pb_mac(%s, t ? xo - x : Sv(0), a); }\n",
            P.ld[0][1][k], P.lvm[0][1][k], (unsigned)P.lxb[0][1][k], cf(P.pb_lb[1][k]).c_str());
    for (int k = P.ln[0][2] - 1; k >= 0; --k)
        put(s, "    { const bool t = (z%d & 0x%xu) != 0u; const uint32_t o = hm::us_at(lh4k ^ 0x%xu) + "
               "hm::r0s_at(t ? (l4 ^ 0x%xu) & 0x3FCu : 0u); const Sv x = *(const Sv *)(Xsb + (t ? o : zo)); "
               "a = hm::pb_mac(%s, t ? xo - x : Sv(0), a); }\n",
            P.ld[0][2][k], P.lvm[0][2][k], (unsigned)P.lxb[0][2][k], (unsigned)P.lxa[0][2][k], cf(P.pb_lb[2][k]).c_str());
    auto xval = [&](int dst) -> const char * {
        for (int e = 0; e < P.nxf; ++e)
            if (P.xf_dst[e] == dst && P.par && P.xf_q[e] == P.H - 1)
                return P.par < 0 ? "(-gx(x_.base - v_))" : "gx(x_.base - v_)";
        return "gx(x_.base + v_)";
    };
    for (int k = P.xn[0][0] - 1; k >= 0; --k)
        put(s, "    { const hm::XSlot x_ = B.xs[%d]; const uint32_t v_ = hm::us_at(lh4 | x_.kofs2) + "
               "hm::r0s_at((l4 ^ 0x%xu) & 0x3FCu); if ((l ^ x_.wm) & x_.vm) a = hm::pb_mac(%s, xo - %s, a); }\n",
            k, (unsigned)P.xxa[0][0][k], cf(P.pb_xb[0][k]).c_str(), xval(k));
    for (int k = P.xn[0][1] - 1; k >= 0; --k)
        put(s, "    { const hm::XSlot x_ = B.xs[%d]; const uint32_t v_ = hm::us_at((lh4 ^ 0x%xu) | x_.kofs2) + "
               "R0own; if ((l ^ x_.wm) & x_.vm) a = hm::pb_mac(%s, xo - %s, a); }\n",
            HM_BLK_SX + k, (unsigned)P.xxa[0][1][k], cf(P.pb_xb[1][k]).c_str(), xval(HM_BLK_SX + k));
    s += "    return hm::blk_high_pb<Sv>(P, B, Xg, r, gx, xo, a);\n}\n};\n";
    return s;
}

// The per-bond row policy with a target table (blk.cu blk_target_table, per-bond form): each
// low slot gathers the row its entry names -- the exchange target, or the row itself when the
// exchange is not allowed, so that h_b (x_i - x_t) is zero without a test -- and cross slots
// take the rank of l ^ 2^p from the table.
std::string gen_row_pb_table(const BlkParams &P, const BondParams &bp) {
    auto hb = [&](int t) { return -bp.jm[t] / 2.0; };
    auto cf = [&](int t) {
        char buf[96];
        snprintf(buf, sizeof buf, "%lldLL, %.9gf", pb_coef(P, hb(t)), hb(t));
        return std::string(buf);
    };
    std::string s;
    s += "struct RowJit {\n"
         "static constexpr int kPad = hm::BLK_XPAD;\n"
         "static constexpr bool kRelUS = false;\n"
         "static constexpr bool kPerBond = true;\n"
         "static constexpr bool kBC = false;\n"
         "template <class Sv>\n"
         "static __device__ __forceinline__ void stage(const hm::BlkParams &, unsigned char *) {}\n"
         "template <class Sv>\n"
         "static __device__ __forceinline__ void block(const hm::BlkParams &, uint32_t) {}\n"
         "template <class Sv, class G>\n"
         "static __device__ __forceinline__ typename hm::PbAcc<Sv>::T sums_pb(const hm::BlkParams &P,\n"
         "        const hm::BlkMeta &B, const unsigned char *Xsb, const unsigned char *Xg, uint32_t l, uint32_t r,\n"
         "        const G &gx, Sv xo) {\n"
         "    (void)l; (void)Xg;\n"
         "    const uint4 *tt = P.tt + (B.lwo + r);\n"
         "    typename hm::PbAcc<Sv>::T a = 0;\n";
    const int nch = (P.tt_n + 7) / 8;
    for (int j = 0; j < nch; ++j) put(s, "    const uint4 q%d = hm::ldg_v4(tt + %uu);\n", j, (unsigned)j * P.tt_stride);
    static const char *comp[4] = {"x", "y", "z", "w"};
    auto entry = [&](int e) {
        char buf[64];
        const int j = e / 8, c = (e % 8) / 2;
        if (e % 2 == 0) snprintf(buf, sizeof buf, "(q%d.%s & 0xFFFFu)", j, comp[c]);
        else snprintf(buf, sizeof buf, "(q%d.%s >> 16)", j, comp[c]);
        return std::string(buf);
    };
    // the table's single slots are the plan's low slots in order (kinds 0..2, class 0)
    int e = 0;
    for (int t = 0; t < 3; ++t)
        for (int k = 0; k < P.ln[0][t]; ++k, ++e)
            put(s, "    a = hm::pb_mac(%s, xo - *(const Sv *)(Xsb + %s), a);\n", cf(P.pb_lb[t][k]).c_str(), entry(e).c_str());
    const int ecross = 2 * P.tt_ntri + P.tt_nsgl;
    auto cross_entry = [&](int t, int k) {
        const int p = __builtin_ctz((unsigned)P.xxa[0][t][k]) - 2 + (t == 1 ? 8 : 0);
        for (int i = 0; i < P.tt_ncross; ++i)
            if (P.tt_cross_p[i] == p) return ecross + i;
        return -1;
    };
    for (int t = 0; t < 2; ++t)
        for (int k = 0; k < P.xn[0][t]; ++k) {
            const int dst = t * HM_BLK_SX + k;
            const char *val = "gx(x_.base + %s)";
            for (int e2 = 0; e2 < P.nxf; ++e2)
                if (P.xf_dst[e2] == dst && P.par && P.xf_q[e2] == P.H - 1)
                    val = P.par < 0 ? "(-gx(x_.base - %s))" : "gx(x_.base - %s)";
            char buf[128];
            snprintf(buf, sizeof buf, val, entry(cross_entry(t, k)).c_str());
            put(s, "    { const hm::XSlot x_ = B.xs[%d]; if ((l ^ x_.wm) & x_.vm) a = hm::pb_mac(%s, xo - %s, a); }\n",
                dst, cf(P.pb_xb[t][k]).c_str(), buf);
        }
    s += "    return hm::blk_high_pb<Sv>(P, B, Xg, r, gx, xo, a);\n}\n};\n";
    return s;
}

// The row policy of a bond-correlation chunk plan (BlkParams::bcmode, per-bond slots):
// every slot of bond k adds g_i (x_i - x_t) to acc[k] when the bond's spins differ at the
// row (blk_sweep.cuh, bc_body).  High bond j reads its block target hbi[j] (~0: parallel).
std::string gen_row_bc(const BlkParams &P, int nbk) {
    std::string s;
    put(s, "struct RowJit {\n"
           "static constexpr int kPad = hm::BLK_XPAD;\n"
           "static constexpr bool kRelUS = false;\n"
           "static constexpr bool kPerBond = false;\n"
           "static constexpr bool kBC = true;\n"
           "static constexpr int kNB = %d;\n", nbk);
    s += "template <class Sv>\n"
         "static __device__ __forceinline__ void stage(const hm::BlkParams &P, unsigned char *dyn) {\n"
         "    hm::RowGeneric<1>::stage<Sv>(P, dyn);\n"
         "}\n"
         "template <class Sv>\n"
         "static __device__ __forceinline__ void block(const hm::BlkParams &, uint32_t) {}\n"
         "template <class Sv, class G>\n"
         "static __device__ __forceinline__ void sums_bc(const hm::BlkParams &P, const hm::BlkMeta &B,\n"
         "        const unsigned char *Xsb, const unsigned char *Xg, uint32_t l, uint32_t r, const G &gx, Sv xo,\n"
         "        ef::df gi, ef::df *acc) {\n"
         "    const uint32_t l4 = l << 2, lh4 = (l >> 8) << 2, lh4k = lh4 | B.kofs;\n"
         "    const uint32_t R0own = hm::r0s_at(l4 & 0x3FCu), R1own = hm::us_at(lh4k);\n"
         "    const uint32_t zo = (uint32_t)((P.max_block + hm::BLK_XPAD - 1) * sizeof(Sv));   // fixed address\n"
         "    (void)R0own; (void)R1own; (void)lh4; (void)gx; (void)zo; (void)Xg;\n";
    std::set<int> ds;
    for (int t = 0; t < 3; ++t)
        for (int k = 0; k < P.ln[0][t]; ++k) ds.insert(P.ld[0][t][k]);
    for (int d : ds) put(s, "    const uint32_t z%d = l ^ (l >> %d);\n", d, d);
    const char *add = "if (t) hm::bc_mac(acc[%d], gi, xo - x); }\n";
    for (int k = 0; k < P.ln[0][0]; ++k) {
        put(s, "    { const bool t = (z%d & 0x%xu) != 0u; const uint32_t o = R1own + hm::r0s_at(t ? (l4 ^ 0x%xu) & 0x3FCu : 0u); "
               "const Sv x = *(const Sv *)(Xsb + (t ? o : zo)); ",
            P.ld[0][0][k], P.lvm[0][0][k], (unsigned)P.lxa[0][0][k]);
        put(s, add, P.pb_lb[0][k]);
    }
    for (int k = 0; k < P.ln[0][1]; ++k) {
        put(s, "    { const bool t = (z%d & 0x%xu) != 0u; const uint32_t o = R0own + hm::us_at(lh4k ^ 0x%xu); "
               "const Sv x = *(const Sv *)(Xsb + (t ? o : zo)); ",
            P.ld[0][1][k], P.lvm[0][1][k], (unsigned)P.lxb[0][1][k]);
        put(s, add, P.pb_lb[1][k]);
    }
    for (int k = 0; k < P.ln[0][2]; ++k) {
        put(s, "    { const bool t = (z%d & 0x%xu) != 0u; const uint32_t o = hm::us_at(lh4k ^ 0x%xu) + "
               "hm::r0s_at(t ? (l4 ^ 0x%xu) & 0x3FCu : 0u); const Sv x = *(const Sv *)(Xsb + (t ? o : zo)); ",
            P.ld[0][2][k], P.lvm[0][2][k], (unsigned)P.lxb[0][2][k], (unsigned)P.lxa[0][2][k]);
        put(s, add, P.pb_lb[2][k]);
    }
    for (int k = 0; k < P.xn[0][0]; ++k)
        put(s, "    { const hm::XSlot x_ = B.xs[%d]; const uint32_t v_ = hm::us_at(lh4 | x_.kofs2) + "
               "hm::r0s_at((l4 ^ 0x%xu) & 0x3FCu); if ((l ^ x_.wm) & x_.vm) "
               "hm::bc_mac(acc[%d], gi, xo - gx(x_.base + v_)); }\n",
            k, (unsigned)P.xxa[0][0][k], P.pb_xb[0][k]);
    for (int k = 0; k < P.xn[0][1]; ++k)
        put(s, "    { const hm::XSlot x_ = B.xs[%d]; const uint32_t v_ = hm::us_at((lh4 ^ 0x%xu) | x_.kofs2) + "
               "R0own; if ((l ^ x_.wm) & x_.vm) hm::bc_mac(acc[%d], gi, xo - gx(x_.base + v_)); }\n",
            HM_BLK_SX + k, (unsigned)P.xxa[0][1][k], P.pb_xb[1][k]);
    for (int j = 0; j < P.nhb; ++j)
        put(s, "    { const uint32_t o = B.hbi[%d]; if (o != 0xFFFFFFFFu) "
               "hm::bc_mac(acc[%d], gi, xo - gx(Xg + (size_t)(o + r) * sizeof(Sv))); }\n",
            j, P.pb_hbb[j]);
    s += "}\n};\n";
    return s;
}

// The row policy of a plan (interface in blk_sweep.cuh), every count, shift and mask a
// literal.  The low bonds with both ends in one byte of the low word take their target
// from per-byte delta tables: the target row of slot s is r + D[b][s], with D = 0 when
// the two spins are parallel (no exchange).  Such a slot then adds the row's own x, and
// every low or cross slot is reported in cnt whether its exchange is allowed or not:
// T_c = 2 acc_c + (ntot_c - 2 cnt_c) x_r turns a reported slot with target r into +x_r,
// the diagonal term of a parallel bond, and one with another target into
// 2 x_target - x_r, as the two terms of Eq. (E-2-1) require.  Bonds across the bytes
// and cross bonds take the own x when not allowed; high bonds are reported only when
// allowed.
//   D0[c][b0][s]: byte offset R0[b0 ^ pat] - R0[b0] (fixed per kernel), 16 bits
//   D1[c][b1][s]: byte offset U[k][b1 ^ pat] - U[k][b1] (rebuilt per block), 32 bits
//   US3[j][b1]: U[k - 1 + j][b1] (per block), for the bonds across bytes and the cross bonds
std::string gen_row(const BlkParams &P, bool &ok) {
    ok = true;
    std::string s;
    const int NC = P.nc;
    int w0 = 1, w1 = 1;
    for (int c = 0; c < NC; ++c) {
        w0 = std::max(w0, (P.ln[c][0] + 7) / 8);
        w1 = std::max(w1, (P.ln[c][1] + 3) / 4);
    }
    if (w0 > 2 || w1 > 4) { ok = false; return s; }
    put(s, "__shared__ uint4 s_D0[%d];\n__shared__ int4 s_D1[%d];\n__shared__ uint32_t s_US3[%d];\n",
        NC * 256 * w0, NC * P.nb1 * w1, 3 * P.nb1);
    s += "__device__ __forceinline__ uint32_t us3_at(uint32_t o) {\n"
         "    return *(const uint32_t *)((const unsigned char *)s_US3 + o);\n}\n";
    s += "struct RowJit {\nstatic constexpr int kPad = 0;\nstatic constexpr bool kRelUS = true;\n"
         "static constexpr bool kPerBond = false;\n"
         "static constexpr bool kBC = false;\n";
    // stage: D0
    s += "template <class Sv>\nstatic __device__ __forceinline__ void stage(const hm::BlkParams &P, unsigned char *) {\n"
         "    const uint8_t *R0g = (const uint8_t *)P.tab + P.off_R0;\n"
         "    const int es = (int)sizeof(Sv);\n"
         "    for (int b0 = threadIdx.x; b0 < 256; b0 += hm::BLK_NT) {\n"
         "        const int r0 = R0g[b0];\n";
    for (int c = 0; c < NC; ++c) {
        put(s, "        {   // class %d\n            int d[%d] = {0};\n", c, 8 * w0);
        for (int k = 0; k < P.ln[c][0]; ++k) {
            const unsigned pat = ((unsigned)P.lxa[c][0][k] >> 2) & 255u;
            put(s, "            d[%d] = __popc(b0 & 0x%xu) == 1 ? (R0g[b0 ^ 0x%x] - r0) * es : 0;\n", k, pat, pat);
        }
        for (int w = 0; w < w0; ++w)
            put(s, "            s_D0[(%d * 256 + b0) * %d + %d] = make_uint4("
                   "(uint32_t)(d[%d] & 0xFFFF) | ((uint32_t)d[%d] << 16), (uint32_t)(d[%d] & 0xFFFF) | ((uint32_t)d[%d] << 16), "
                   "(uint32_t)(d[%d] & 0xFFFF) | ((uint32_t)d[%d] << 16), (uint32_t)(d[%d] & 0xFFFF) | ((uint32_t)d[%d] << 16));\n",
                c, w0, w, 8 * w, 8 * w + 1, 8 * w + 2, 8 * w + 3, 8 * w + 4, 8 * w + 5, 8 * w + 6, 8 * w + 7);
        s += "        }\n";
    }
    s += "    }\n}\n";
    // block: US3 and D1
    put(s, "template <class Sv>\nstatic __device__ __forceinline__ void block(const hm::BlkParams &P, uint32_t k) {\n"
           "    const uint16_t *Ug = (const uint16_t *)((const unsigned char *)P.tab + P.off_U);\n"
           "    const int es = (int)sizeof(Sv);\n"
           "    for (int i = threadIdx.x; i < %d; i += hm::BLK_NT) {\n"
           "        const int j = i / %d, b1 = i %% %d, kk = (int)k - 1 + j;\n"
           "        s_US3[i] = (kk >= 0 && kk <= %d) ? (uint32_t)Ug[kk * %d + b1] * (uint32_t)es : 0u;\n"
           "    }\n"
           "    for (int b1 = threadIdx.x; b1 < %d; b1 += hm::BLK_NT) {\n"
           "        const uint16_t *Uk = Ug + k * %d;\n"
           "        const int u0 = Uk[b1];\n",
        3 * P.nb1, P.nb1, P.nb1, P.K, P.nb1, P.nb1, P.nb1);
    for (int c = 0; c < NC; ++c) {
        put(s, "        {   // class %d\n            int d[%d] = {0};\n", c, 4 * w1);
        for (int k = 0; k < P.ln[c][1]; ++k) {
            const unsigned pat = ((unsigned)P.lxb[c][1][k] >> 2);
            put(s, "            d[%d] = __popc(b1 & 0x%xu) == 1 ? (Uk[b1 ^ 0x%x] - u0) * es : 0;\n", k, pat, pat);
        }
        for (int w = 0; w < w1; ++w)
            put(s, "            s_D1[(%d * %d + b1) * %d + %d] = make_int4(d[%d], d[%d], d[%d], d[%d]);\n", c, P.nb1, w1, w,
                4 * w, 4 * w + 1, 4 * w + 2, 4 * w + 3);
        s += "        }\n";
    }
    s += "    }\n}\n";
    // sums
    s += "template <class Sv, class G>\n"
         "static __device__ __forceinline__ void sums(const hm::BlkParams &P, const hm::BlkMeta &B,\n"
         "        const unsigned char *Xsb, const unsigned char *Xg, uint32_t l, uint32_t r, const G &gx, Sv xo,\n"
         "        Sv *acc, int *cnt) {\n"
         "    const uint32_t b0 = l & 255u, b1 = l >> 8, rb = r * (uint32_t)sizeof(Sv);\n"
         "    const uint32_t l4 = l << 2, lh4 = b1 << 2;\n"
         "    (void)b0; (void)b1; (void)l4; (void)lh4; (void)xo; (void)gx;\n";
    std::set<int> ds;
    bool need_r0own = false;
    for (int c = 0; c < NC; ++c) {
        for (int k = 0; k < P.ln[c][2]; ++k) ds.insert(P.ld[c][2][k]);
        if (P.xn[c][1] > 0) need_r0own = true;
    }
    for (int d : ds) put(s, "    const uint32_t z%d = l ^ (l >> %d);\n", d, d);
    if (need_r0own) s += "    const uint32_t R0own = hm::r0s_at(l4 & 0x3FCu);\n";
    s += "#define XS(o) (*(const Sv *)(Xsb + (o)))\n";
    for (int c = 0; c < NC; ++c) {
        put(s, "    {   // class %d\n        Sv a = Sv(0);\n", c);
        for (int w = 0; w < w0 && w * 8 < P.ln[c][0]; ++w) {
            put(s, "        { const uint4 q = s_D0[(%d * 256 + b0) * %d + %d];\n", c, w0, w);
            const char *fld[4] = {"x", "y", "z", "w"};
            for (int k = 8 * w; k < std::min(P.ln[c][0], 8 * w + 8); ++k) {
                const int j = k - 8 * w;
                if (j % 2 == 0) put(s, "          a += XS(rb + (int)(short)(q.%s & 0xFFFFu));\n", fld[j / 2]);
                else put(s, "          a += XS(rb + ((int)q.%s >> 16));\n", fld[j / 2]);
            }
            s += "        }\n";
        }
        for (int w = 0; w < w1 && w * 4 < P.ln[c][1]; ++w) {
            put(s, "        { const int4 q = s_D1[(%d * %d + b1) * %d + %d];\n", c, P.nb1, w1, w);
            const char *fld[4] = {"x", "y", "z", "w"};
            for (int k = 4 * w; k < std::min(P.ln[c][1], 4 * w + 4); ++k)
                put(s, "          a += XS(rb + q.%s);\n", fld[k - 4 * w]);
            s += "        }\n";
        }
        for (int k = 0; k < P.ln[c][2]; ++k)
            put(s, "        { const uint32_t t = z%d & 0x%xu; const uint32_t v = us3_at(%uu | (lh4 ^ 0x%xu)) + "
                   "hm::r0s_at((l4 ^ 0x%xu) & 0x3FCu); a += XS(t ? v : rb); }\n",
                P.ld[c][2][k], P.lvm[c][2][k], 1u << P.kshift, (unsigned)P.lxb[c][2][k], (unsigned)P.lxa[c][2][k]);
        for (int k = 0; k < P.xn[c][0]; ++k)
            put(s, "        { const hm::XSlot x_ = B.xs[%d]; const uint32_t t = (l ^ x_.wm) & x_.vm; "
                   "const uint32_t v = us3_at(x_.kofs2 | lh4) + hm::r0s_at((l4 ^ 0x%xu) & 0x3FCu); "
                   "a += t ? gx(x_.base + v) : xo; }\n",
                (2 * c) * HM_BLK_SX + k, (unsigned)P.xxa[c][0][k]);
        for (int k = 0; k < P.xn[c][1]; ++k)
            put(s, "        { const hm::XSlot x_ = B.xs[%d]; const uint32_t t = (l ^ x_.wm) & x_.vm; "
                   "const uint32_t v = us3_at(x_.kofs2 | (lh4 ^ 0x%xu)) + R0own; a += t ? gx(x_.base + v) : xo; }\n",
                (2 * c + 1) * HM_BLK_SX + k, (unsigned)P.xxa[c][1][k]);
        put(s, "        a += hm::blk_high_sum<Sv>(B, %d, Xg, r, gx);\n", c);
        put(s, "        acc[%d] = a;\n        cnt[%d] = %d + (B.he[%d] - B.hs[%d]);\n    }\n", c, c,
            P.ln[c][0] + P.ln[c][1] + P.ln[c][2] + P.xn[c][0] + P.xn[c][1], c, c);
    }
    s += "#undef XS\n}\n};\n";
    return s;
}

// The s = 1 row terms of the low sites of plan P written out (s1_sweep.cuh): every rank
// table entry of the row is loaded first (coalesced: consecutive rows read consecutive
// entries, both directions of a pair or site in one word), then each low bond adds its
// diagonal term and its exchanges gathered from the staged block, and each low site with
// cross bonds its share of the diagonal and the gathers from the blocks one unit of digit
// sum away.  f64: integer couplings C_b and one exact int128 product per bond of C_b and
// the sum of its (up to two) gathered values (row64), else float -J_b (row32).
std::string gen_s1_row(const S1Plan &P, bool f64) {
    std::string s = "#include \"s1_sweep.cuh\"\nstruct S1Row {\n";
    if (f64)
        s += "static __device__ __forceinline__ void row64(uint32_t l, const long long *Xs,\n"
             "        const long long *__restrict__ x, const uint32_t *__restrict__ rl, const uint32_t *__restrict__ rx,\n"
             "        const uint32_t *cb, const long long *cc, long long &dg, __int128 &a) {\n";
    else
        s += "static __device__ __forceinline__ void row32(uint32_t l, const float *Xs, const float *__restrict__ x,\n"
             "        const uint32_t *__restrict__ rl, const uint32_t *__restrict__ rx, const uint32_t *cb,\n"
             "        const float *cc, float &dg, float &acc) {\n";
    bool used[S1_MAXK] = {}, crs[S1_MAXK] = {};
    for (int j = 0; j < P.nlo; ++j) used[P.lo_p[j]] = used[P.lo_q[j]] = true;
    for (int j = 0; j < P.ncr; ++j) used[P.cr_p[j]] = crs[P.cr_p[j]] = true;
    const unsigned nl = (unsigned)P.nlw;
    for (int j = 0; j < P.nlo; ++j) {
        const int p = P.lo_p[j], q = P.lo_q[j], pi = q * (q - 1) / 2 + p;
        put(s, "    const uint32_t L%d = rl[%uu];\n", j, (unsigned)pi * nl);
    }
    for (int p = 0; p < P.K; ++p)
        if (crs[p]) put(s, "    const uint32_t X%d = rx[%uu];\n", p, (unsigned)p * nl);
    for (int p = 0; p < P.K; ++p)
        if (used[p]) {
            if (f64) put(s, "    const int m%d = 1 - (int)((l >> %d) & 3u);\n", p, 2 * p);
            else put(s, "    const float m%d = (float)(1 - (int)((l >> %d) & 3u));\n", p, 2 * p);
        }
    for (int j = 0; j < P.nlo; ++j) {
        const int p = P.lo_p[j], q = P.lo_q[j];
        put(s, "    { const uint32_t t0 = L%d & 0xFFFFu, t1 = L%d >> 16;\n", j, j);
        if (f64) {
            const long long c = P.lo_c[j];
            put(s, "      dg += (long long)(m%d * m%d) * (%lldLL);\n", p, q, c);
            // both directions of the bond summed first: one 128-bit product per bond
            s += "      long long v = t0 != 0xFFFFu ? Xs[t0] : 0ll;\n      if (t1 != 0xFFFFu) v += Xs[t1];\n";
            put(s, "      a += (__int128)v * (%lldLL);\n", c);
        } else {
            const double c = (double)P.lo_j[j];
            put(s, "      dg = fmaf(%af, m%d * m%d, dg);\n", c, p, q);
            for (int d = 0; d < 2; ++d) put(s, "      if (t%d != 0xFFFFu) acc = fmaf(%af, Xs[t%d], acc);\n", d, c, d);
        }
        s += "    }\n";
    }
    for (int p = 0; p < P.K; ++p) {
        if (!crs[p]) continue;
        put(s, "    { const uint32_t t0 = X%d & 0xFFFFu, t1 = X%d >> 16;\n", p, p);
        if (f64) put(s, "      dg += (long long)m%d * cc[%d];\n", p, p);
        else put(s, "      dg = fmaf(cc[%d], m%d, dg);\n", p, p);
        for (int j = 0; j < P.ncr; ++j) {
            if (P.cr_p[j] != p) continue;
            put(s, "      { const uint32_t b0 = cb[%d], b1 = cb[%d];\n", 2 * j, 2 * j + 1);
            if (f64) {
                s += "        long long v = t0 != 0xFFFFu && b0 != 0xFFFFFFFFu ? __ldg(x + (b0 + t0)) : 0ll;\n"
                     "        if (t1 != 0xFFFFu && b1 != 0xFFFFFFFFu) v += __ldg(x + (b1 + t1));\n";
                put(s, "        a += (__int128)v * (%lldLL);\n", P.cr_c[j]);
            } else {
                for (int d = 0; d < 2; ++d)
                    put(s, "        if (t%d != 0xFFFFu && b%d != 0xFFFFFFFFu) acc = fmaf(%af, __ldg(x + (b%d + t%d)), acc);\n",
                        d, d, (double)P.cr_j[j], d, d);
            }
            s += "      }\n";
        }
        s += "    }\n";
    }
    s += "}\n};\n";
    return s;
}

int compile(const std::string &src, const char *name, int device, const void **out) {
    // HM_JIT_DUMP=<dir>: keep each generated source as <dir>/<kernel>_<n>.cu (for offline
    // compilation and register reports)
    if (const char *d = getenv("HM_JIT_DUMP")) {
        static int seq = 0;
        char path[4096];
        snprintf(path, sizeof path, "%s/%s_%d.cu", d, name, seq++);
        if (FILE *f = fopen(path, "w")) { fputs(src.c_str(), f); fclose(f); }
    }
    nvrtcProgram prog;
    if (g_nv.create(&prog, src.c_str(), "hm_jit.cu", (int)(sizeof kJitHeaderNames / sizeof *kJitHeaderNames),
                    kJitHeaderTexts, kJitHeaderNames) != NVRTC_SUCCESS)
        return 1;
    const char *opts[] = {"--gpu-architecture=sm_103a", "-std=c++17", "--device-int128", "-lineinfo",
                          "--fmad=true", "--ptxas-options=-v"};
    const int nopt = (int)(sizeof opts / sizeof *opts) - (verbose() ? 0 : 1);   // ptxas report when verbose
    const nvrtcResult rc = g_nv.compile(prog, nopt, opts);
    if (rc != NVRTC_SUCCESS || verbose()) {
        size_t n = 0;
        g_nv.log_size(prog, &n);
        std::string log(n, '\0');
        if (n) g_nv.log(prog, &log[0]);
        if (rc != NVRTC_SUCCESS || verbose()) fprintf(stderr, "[hm jit] %s: %s\n", name, log.c_str());
    }
    if (rc != NVRTC_SUCCESS) { g_nv.destroy(&prog); return 1; }
    size_t n = 0;
    g_nv.cubin_size(prog, &n);
    std::vector<char> bin(n);
    g_nv.cubin(prog, bin.data());
    g_nv.destroy(&prog);
    cudaLibrary_t lib;
    if (cudaLibraryLoadData(&lib, bin.data(), nullptr, nullptr, 0, nullptr, nullptr, 0) != cudaSuccess) {
        cudaGetLastError();
        return 1;
    }
    cudaKernel_t k;
    if (cudaLibraryGetKernel(&k, lib, name) != cudaSuccess) { cudaGetLastError(); return 1; }
    (void)device;
    *out = (const void *)k;
    return 0;
}

}  // namespace

// Kernel of the Lanczos product for plan P (dtype HM_F64: k_blk_lz64_jit, HM_F32:
// k_blk_lz32_jit), compiled on first use and cached for the process.  Returns 0 and the
// handle (usable with cudaLaunchKernel / cudaFuncSetAttribute), or 1 when the generic
// kernel has to serve.
// source of the row policy for plan P: per-bond, per-byte delta tables, or slots
static bool jit_row_source(const BlkParams &P, const BondParams &bp, std::string *src, bool *delta) {
    bool gen_ok = true;
    const char *rowk = getenv("HM_JIT_ROW");
    *delta = !P.perbond && rowk && strcmp(rowk, "delta") == 0 && !P.par;   // no spin-flip or per-bond form
    *src = std::string("#include \"blk_sweep.cuh\"\n") +
           (P.perbond ? gen_row_pb(P, bp) : *delta ? gen_row(P, gen_ok) : P.tt ? gen_row_table(P) : gen_row_slots(P));
    return gen_ok;
}

// compiles (or finds) kernel `name` of source src for the current device
static int jit_get(const std::string &src, const char *name, int dev, int pad, const void **kern) {
    const std::string key = std::to_string(dev) + "\n" + src;
    std::lock_guard<std::mutex> lk(g_mu);
    auto it = g_cache.find(key);
    if (it != g_cache.end()) { *kern = it->second; return 0; }
    if (g_failed.count(key)) return 1;
    if (!load_nvrtc()) {
        if (verbose()) fprintf(stderr, "[hm jit] %s\n", g_nv.why.c_str());
        return 1;
    }
    const void *k = nullptr;
    if (compile(src, name, dev, &k) != 0) { g_failed.insert(key); return 1; }
    g_cache.emplace(key, k);
    g_pad[k] = pad;
    *kern = k;
    return 0;
}

// y = H x kernel (matvec API) for a per-bond plan: k_blk_matvec_jit, one vector, dtype
// HM_F64 (binary64 x, E = its largest exponent field in Eptr) or HM_F32
int jit_mv_kernel(const BlkParams &P, int dtype, const BondParams &bp, const void **kern) {
    const char *env = getenv("HM_JIT");
    if ((env && env[0] == '0') || !P.rows_ok || !P.perbond) return 1;
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess) { cudaGetLastError(); return 1; }
    std::string src;
    bool delta = false;
    if (!jit_row_source(P, bp, &src, &delta)) return 1;
    const char *T = dtype == HM_F64 ? "double" : "float";
    put(src,
        "extern \"C\" __global__ void __launch_bounds__(512, 3) k_blk_matvec_jit(hm::BlkParams P,\n"
        "        const %s *__restrict__ x, %s *__restrict__ y, const int *__restrict__ Eptr) {\n"
        "    hm::matvec_body<%s, 1, RowJit>(P, x, y, Eptr);\n}\n", T, T, T);
    return jit_get(src, "k_blk_matvec_jit", dev, BLK_XPAD, kern);
}

// bond-correlation kernel of a chunk plan (bcmode) with nbk bonds: k_blk_bc_jit, dtype
// HM_F64 (binary64 x and g, E = largest exponent field of x in Eptr) or HM_F32
int jit_bc_kernel(const BlkParams &P, int dtype, int nbk, const void **kern) {
    const char *env = getenv("HM_JIT");
    if ((env && env[0] == '0') || !P.rows_ok || !P.bcmode) return 1;
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess) { cudaGetLastError(); return 1; }
    std::string src = "#include \"blk_sweep.cuh\"\n" + gen_row_bc(P, nbk);
    const char *T = dtype == HM_F64 ? "double" : "float";
    put(src,
        "extern \"C\" __global__ void __launch_bounds__(512, 2) k_blk_bc_jit(hm::BlkParams P,\n"
        "        const %s *__restrict__ x, const %s *__restrict__ g, const int *__restrict__ Eptr,\n"
        "        double *__restrict__ part) {\n"
        "    hm::bc_body<%s, RowJit>(P, x, g, Eptr, part);\n}\n", T, T, T);
    return jit_get(src, "k_blk_bc_jit", dev, BLK_XPAD, kern);
}

// split = 1 / 2: the passes of the split FP64 product (k_blk_lz64a_jit / k_blk_lz64b_jit,
// plans of the near and of the far bonds; blk_sweep.cuh, lz64_body)
int jit_lz_kernel(const BlkParams &P, int dtype, const BondParams &bp, const void **kern, int split) {
    const char *env = getenv("HM_JIT");
    if (env && env[0] == '0') return 1;
    if (!P.rows_ok) return 1;
    if (split && (dtype != HM_F64 || !P.iratio || !P.g0_pow2 || P.perbond || P.par)) return 1;
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess) { cudaGetLastError(); return 1; }
    std::string src;
    bool delta = false;
    if (!jit_row_source(P, bp, &src, &delta)) return 1;
    const bool f64 = dtype == HM_F64;
    const int nc = P.nc == 1 ? 1 : (P.nc == 2 ? 2 : 4);
    const char *name = !f64 ? "k_blk_lz32_jit" : split == 1 ? "k_blk_lz64a_jit" : split == 2 ? "k_blk_lz64b_jit"
                                                                                         : "k_blk_lz64_jit";
    // resident CTAs per SM the register budget is cut for (3: 40 registers a thread, 2: 64);
    // HM_JIT_CTAS overrides the default
    int ctas = 3;
    if (const char *e = getenv("HM_JIT_CTAS")) ctas = atoi(e) == 2 ? 2 : 3;
    if (f64)
        put(src,
            "extern \"C\" __global__ void __launch_bounds__(512, %d) %s(hm::BlkParams P,\n"
            "        const long long *__restrict__ Xc, unsigned long long *__restrict__ Y, hm::LzScalars *S, int pc,\n"
            "        double *__restrict__ part) {\n"
            "    hm::lz64_body<%d, %s, RowJit, %d>(P, Xc, Y, S, pc, part);\n}\n",
            ctas, name, nc, P.iratio && !P.perbond ? "true" : "false", split);
    else
        put(src,
            "extern \"C\" __global__ void __launch_bounds__(512, %d) k_blk_lz32_jit(hm::BlkParams P,\n"
            "        const float *__restrict__ qc, float *__restrict__ qp, hm::LzScalars *S, double *__restrict__ part) {\n"
            "    hm::lz32_body<%d, RowJit>(P, qc, qp, S, part);\n}\n",
            ctas, nc);
    return jit_get(src, name, dev, delta ? 0 : BLK_XPAD, kern);
}

int jit_s1_kernel(const S1Plan &P, int mode, const void **kern) {
    if (mode < 0 || mode > 2) return 1;
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess) { cudaGetLastError(); return 1; }
    std::string src = gen_s1_row(P, mode == 2);
    static const char *const names[3] = {"k_s1_mv_jit", "k_s1_lz32_jit", "k_s1_lz64_jit"};
    // FP32: resident CTAs per SM the register budget is cut for (HM_S1_CTAS: 2 or 3)
    int ctas = 3;
    if (const char *e = getenv("HM_S1_CTAS")) ctas = atoi(e) == 2 ? 2 : 3;
    if (mode == 0)
        put(src, "extern \"C\" __global__ void __launch_bounds__(512, %d) k_s1_mv_jit(hm::S1Plan P,\n"
                 "        const float *__restrict__ x, float *__restrict__ y) {\n"
                 "    hm::s1j_body32<S1Row, false>(P, x, y, nullptr, nullptr);\n}\n", ctas);
    else if (mode == 1)
        put(src, "extern \"C\" __global__ void __launch_bounds__(512, %d) k_s1_lz32_jit(hm::S1Plan P,\n"
                 "        const float *__restrict__ qc, float *__restrict__ qp, const hm::LzScalars *__restrict__ S,\n"
                 "        double *__restrict__ part) {\n"
                 "    hm::s1j_body32<S1Row, true>(P, qc, qp, S, part);\n}\n", ctas);
    else
        src += "extern \"C\" __global__ void __launch_bounds__(512, 2) k_s1_lz64_jit(hm::S1Plan P,\n"
               "        const long long *__restrict__ Xc, unsigned long long *__restrict__ Y,\n"
               "        const hm::LzScalars *__restrict__ S, int pc, double *__restrict__ part) {\n"
               "    hm::s1j_body64<S1Row>(P, Xc, Y, S, pc, part);\n}\n";
    return jit_get(src, names[mode], dev, 0, kern);
}

int jit_pad(const void *kern) {
    if (!kern) return BLK_XPAD;
    std::lock_guard<std::mutex> lk(g_mu);
    auto it = g_pad.find(kern);
    return it == g_pad.end() ? BLK_XPAD : it->second;
}

}  // namespace hm
