// jit.cu -- the s = 1/2 Lanczos products specialised to one bond list at run time.
//
// The generic block kernels (blk.cu) read every bond slot from the kernel parameters and
// enter the runs of slots through switches.  Here the slots of a plan are written out as
// straight-line code with their positions and masks as literals, the result is compiled
// for sm_103a with NVRTC and loaded with cudaLibraryLoadData.  Both variants run the
// same bodies (blk_sweep.cuh) and form the same exact integer sums, so their outputs
// agree bit for bit; the generic kernel stays the fallback when NVRTC is not available
// (HM_JIT=0 selects it on purpose).
#include <dlfcn.h>
#include <nvrtc.h>

#include <cstdarg>
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <map>
#include <mutex>
#include <set>
#include <string>
#include <vector>

#include "blk.cuh"
#include "blk_sweep.cuh"
#include "jit_embed.inc"   // kJitHeaderNames / kJitHeaderTexts: the .cuh files above, as text

#ifndef HM_CUDA_LIBDIR
#define HM_CUDA_LIBDIR "/usr/local/cuda/lib64"
#endif

namespace hm {
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
    char buf[512];
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(buf, sizeof buf, fmt, ap);
    va_end(ap);
    s += buf;
}

// The row policy of a plan: the slots of RowGeneric (blk_sweep.cuh) with every count,
// shift and mask a literal, in RowGeneric's order (each run from its last slot down, so
// FP32 sums round the same way).  Failed exchanges read x too (the staged rows are padded, so
// the address stays inside the buffer) and add under the test's predicate.
std::string gen_row(const BlkParams &P) {
    std::string s;
    s += "struct RowJit {\n"
         "template <class Sv, class G>\n"
         "static __device__ __forceinline__ void sums(const hm::BlkParams &P, const hm::BlkMeta &B,\n"
         "        const unsigned char *Xsb, uint32_t l, uint32_t r, const G &gx, Sv *acc, int *cnt) {\n"
         "    const uint32_t l4 = l << 2, lh4 = (l >> 8) << 2, lh4k = lh4 | B.kofs;\n"
         "    const uint32_t R0own = hm::r0s_at(l4 & 0x3FCu), R1own = hm::us_at(lh4k);\n"
         "    const uint32_t rb = r * (uint32_t)sizeof(Sv);\n"
         "    (void)R0own; (void)R1own; (void)lh4; (void)gx;\n";
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
            put(s, "        { const Sv v = *(const Sv *)(Xsb + R1own + hm::r0s_at((l4 ^ 0x%xu) & 0x3FCu)); "
                   "if (z%d & 0x%xu) a += v; }\n",
                (unsigned)P.lxa[c][0][k], P.ld[c][0][k], P.lvm[c][0][k]);
        for (int k = P.ln[c][1] - 1; k >= 0; --k)
            put(s, "        { const Sv v = *(const Sv *)(Xsb + R0own + hm::us_at(lh4k ^ 0x%xu)); "
                   "if (z%d & 0x%xu) a += v; }\n",
                (unsigned)P.lxb[c][1][k], P.ld[c][1][k], P.lvm[c][1][k]);
        for (int k = P.ln[c][2] - 1; k >= 0; --k)
            put(s, "        { const Sv v = *(const Sv *)(Xsb + hm::us_at(lh4k ^ 0x%xu) + "
                   "hm::r0s_at((l4 ^ 0x%xu) & 0x3FCu)); if (z%d & 0x%xu) a += v; }\n",
                (unsigned)P.lxb[c][2][k], (unsigned)P.lxa[c][2][k], P.ld[c][2][k], P.lvm[c][2][k]);
        for (int g = P.lgn[c] - 1; g >= 0; --g) put(s, "        m += __popc(z%d & 0x%xu);\n", P.lgd[c][g], P.lgm[c][g]);
        for (int k = P.xn[c][0] - 1; k >= 0; --k)
            put(s, "        { const hm::XSlot x_ = B.xs[%d]; const uint32_t v_ = hm::us_at(lh4 | x_.kofs2) + "
                   "hm::r0s_at((l4 ^ 0x%xu) & 0x3FCu); if ((l ^ x_.wm) & x_.vm) { a += gx(x_.base + v_); ++m; } }\n",
                (2 * c) * HM_BLK_SX + k, (unsigned)P.xxa[c][0][k]);
        for (int k = P.xn[c][1] - 1; k >= 0; --k)
            put(s, "        { const hm::XSlot x_ = B.xs[%d]; const uint32_t v_ = hm::us_at((lh4 ^ 0x%xu) | x_.kofs2) + "
                   "R0own; if ((l ^ x_.wm) & x_.vm) { a += gx(x_.base + v_); ++m; } }\n",
                (2 * c + 1) * HM_BLK_SX + k, (unsigned)P.xxa[c][1][k]);
        put(s, "        const int e0 = B.hs[%d], e1 = B.hs[%d];\n", c, c + 1);
        s += "        int e = e0;\n"
             "        for (; e + 4 <= e1; e += 4) {\n"
             "            const Sv v0 = gx(B.hb[e] + rb), v1 = gx(B.hb[e + 1] + rb);\n"
             "            const Sv v2 = gx(B.hb[e + 2] + rb), v3 = gx(B.hb[e + 3] + rb);\n"
             "            a += (v0 + v1) + (v2 + v3);\n"
             "        }\n"
             "        for (; e < e1; ++e) a += gx(B.hb[e] + rb);\n";
        put(s, "        acc[%d] = a;\n        cnt[%d] = m + (e1 - e0);\n    }\n", c, c);
    }
    s += "}\n};\n";
    return s;
}

int compile(const std::string &src, const char *name, int device, const void **out) {
    nvrtcProgram prog;
    if (g_nv.create(&prog, src.c_str(), "hm_jit.cu", (int)(sizeof kJitHeaderNames / sizeof *kJitHeaderNames),
                    kJitHeaderTexts, kJitHeaderNames) != NVRTC_SUCCESS)
        return 1;
    const char *opts[] = {"--gpu-architecture=sm_103a", "-std=c++17", "--device-int128", "-lineinfo",
                          "--fmad=true"};
    const nvrtcResult rc = g_nv.compile(prog, (int)(sizeof opts / sizeof *opts), opts);
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
int jit_lz_kernel(const BlkParams &P, int dtype, const void **kern) {
    const char *env = getenv("HM_JIT");
    if (env && env[0] == '0') return 1;
    if (!P.rows_ok) return 1;
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess) { cudaGetLastError(); return 1; }
    std::string src = "#include \"blk_sweep.cuh\"\n" + gen_row(P);
    const bool f64 = dtype == HM_F64;
    const int nc = P.nc == 1 ? 1 : (P.nc == 2 ? 2 : 4);
    const char *name = f64 ? "k_blk_lz64_jit" : "k_blk_lz32_jit";
    if (f64)
        put(src,
            "extern \"C\" __global__ void __launch_bounds__(512, 3) k_blk_lz64_jit(hm::BlkParams P,\n"
            "        const long long *__restrict__ Xc, const long long *__restrict__ Xp,\n"
            "        unsigned long long *__restrict__ Y, hm::LzScalars *S, int pc, double *__restrict__ part) {\n"
            "    hm::lz64_body<%d, %s, RowJit>(P, Xc, Xp, Y, S, pc, part);\n}\n",
            nc, P.iratio ? "true" : "false");
    else
        put(src,
            "extern \"C\" __global__ void __launch_bounds__(512, 3) k_blk_lz32_jit(hm::BlkParams P,\n"
            "        const float *__restrict__ qc, float *__restrict__ qp, hm::LzScalars *S, double *__restrict__ part) {\n"
            "    hm::lz32_body<%d, RowJit>(P, qc, qp, S, part);\n}\n",
            nc);
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
    *kern = k;
    return 0;
}

}  // namespace hm
