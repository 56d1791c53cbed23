// sectors.cu -- the lowest energy of every magnetisation sector H(M) of one bond list: the
// curve E0(M) the applications of the Lanczos machinery work with (Sec. 1), from one
// FP64 (or FP32) Lanczos run per sector on the sector coding of Sec. 3.  All runs are the
// branches of one captured CUDA graph, launched once: no host round trip per sector, and the
// many small sectors run side by side on the GPU.
#include <algorithm>
#include <vector>

#include "hm_internal.cuh"

namespace hm {

size_t lz_run_workspace(const hm_basis *b, int dtype, int steps);
int lz_branches(const std::vector<const hm_basis *> &bases, int n_bonds, const int32_t *u, const int32_t *v,
                const double *J, const std::vector<uint64_t> &seeds, int steps, int dtype, unsigned char *work,
                const std::vector<size_t> &offs, double *out, cudaStream_t st);

// start vector key of sector A: output #(A 2^20) of the caller's SplitMix64 seed, the
// key the finite-temperature driver gives the first vector of sector A
static uint64_t sector_seed(uint64_t seed, int A) { return sm64(seed, (uint64_t)A << 20); }

static size_t al256s(size_t x) { return (x + 255) & ~(size_t)255; }

// the sectors' bases (caller frees them) and the workspace layout: run A at offs[A], the
// per-run results (3 doubles each) at *res
static int sector_layout(int n_sites, int two_s, int steps, int dtype, std::vector<hm_basis *> *bases,
                         std::vector<size_t> *offs, size_t *res, size_t *total) {
    const int nsec = two_s * n_sites + 1;
    size_t o = 0;
    for (int A = 0; A < nsec; ++A) {
        hm_basis *b = nullptr;
        const int rc = basis_build(n_sites, two_s, two_s * n_sites - 2 * A, &b);
        if (rc < 0) return rc;
        bases->push_back(b);
        offs->push_back(o);
        o += al256s(lz_run_workspace(b, dtype, steps));
    }
    *res = o;
    *total = o + al256s((size_t)nsec * 3 * sizeof(double));
    return HM_OK;
}

static void free_bases(std::vector<hm_basis *> &bases) {
    for (hm_basis *b : bases) basis_free(b);
    bases.clear();
}

}  // namespace hm

using namespace hm;

extern "C" int sector_ground_energies_workspace(int n_sites, int two_s, int steps, int dtype, size_t *bytes) {
    if (!bytes) return fail(HM_EINVAL, "NULL argument");
    *bytes = 0;
    if (n_sites < 1 || two_s < 1) return fail(HM_EINVAL, "n_sites and two_s must be positive");
    if (dtype != HM_F64 && dtype != HM_F32) return fail(HM_EINVAL, "bad dtype");
    if (steps < 1 || steps > 100000) return fail(HM_EINVAL, "steps must be in 1..100000");
    std::vector<hm_basis *> bases;
    std::vector<size_t> offs;
    size_t res = 0, total = 0;
    const int rc = sector_layout(n_sites, two_s, steps, dtype, &bases, &offs, &res, &total);
    free_bases(bases);
    HM_TRY(rc);
    *bytes = total;
    return HM_OK;
}

extern "C" int sector_ground_energies(int n_sites, int two_s, int n_bonds, const int32_t *u, const int32_t *v,
                                      const double *J, int steps, uint64_t seed, int dtype, void *work,
                                      size_t work_bytes, double *e0, int *steps_done, void *stream) {
    if (!e0) return fail(HM_EINVAL, "e0 is NULL");
    if (n_sites < 1 || two_s < 1) return fail(HM_EINVAL, "n_sites and two_s must be positive");
    if (dtype != HM_F64 && dtype != HM_F32) return fail(HM_EINVAL, "bad dtype");
    if (steps < 1 || steps > 100000) return fail(HM_EINVAL, "steps must be in 1..100000");
    HM_TRY(bonds_check(n_sites, n_bonds, u, v, J));
    const int nsec = two_s * n_sites + 1;
    std::vector<hm_basis *> bases;
    std::vector<size_t> offs;
    size_t res = 0, total = 0;
    int rc = sector_layout(n_sites, two_s, steps, dtype, &bases, &offs, &res, &total);
    if (rc == HM_OK && (!work || work_bytes < total || ((uintptr_t)work & 255)))
        rc = fail(HM_EWORKSPACE, "sector_ground_energies needs %zu workspace bytes, 256-byte aligned", total);
    std::vector<double> out((size_t)nsec * 3, 0.0);
    if (rc == HM_OK) {
        std::vector<const hm_basis *> cb(bases.begin(), bases.end());
        std::vector<uint64_t> seeds(nsec);
        for (int A = 0; A < nsec; ++A) seeds[A] = sector_seed(seed, A);
        unsigned char *w = (unsigned char *)work;
        cudaStream_t st = as_stream(stream);
        rc = lz_branches(cb, n_bonds, u, v, J, seeds, steps, dtype, w, offs, (double *)(w + res), st);
        if (rc == HM_OK) {
            cudaError_t e = cudaMemcpyAsync(out.data(), w + res, out.size() * sizeof(double), cudaMemcpyDeviceToHost, st);
            if (e == cudaSuccess) e = cudaStreamSynchronize(st);
            if (e != cudaSuccess) rc = cuda_fail(e, "sector results");
        }
    }
    free_bases(bases);
    HM_TRY(rc);
    for (int A = 0; A < nsec; ++A) {
        const int status = (int)out[3 * A + 2];
        if (status < 0) return fail(status, "sector A = %d: Lanczos start vector has zero norm", A);
        e0[A] = out[3 * A];
        if (steps_done) steps_done[A] = (int)out[3 * A + 1];
    }
    return HM_OK;
}
