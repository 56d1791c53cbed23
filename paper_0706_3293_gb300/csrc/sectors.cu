// sectors.cu -- the lowest energy of every magnetisation sector H(M) of one bond list: the
// curve E0(M) the applications of the Lanczos machinery work with (Sec. 1), from one
// FP64 (or FP32) Lanczos run per sector on the sector coding of Sec. 3.
#include <algorithm>
#include <vector>

#include "hm_internal.cuh"

namespace hm {

// start vector key of sector A: output #(A 2^20) of the caller's SplitMix64 seed, the
// key the finite-temperature driver gives the first vector of sector A
static uint64_t sector_seed(uint64_t seed, int A) { return sm64(seed, (uint64_t)A << 20); }

}  // namespace hm

using namespace hm;

extern "C" int sector_ground_energies_workspace(int n_sites, int two_s, int steps, int dtype, size_t *bytes) {
    if (!bytes) return fail(HM_EINVAL, "NULL argument");
    *bytes = 0;
    if (n_sites < 1 || two_s < 1) return fail(HM_EINVAL, "n_sites and two_s must be positive");
    const int nsec = two_s * n_sites + 1;
    for (int A = 0; A < nsec; ++A) {
        hm_basis *b = nullptr;
        HM_TRY(basis_build(n_sites, two_s, two_s * n_sites - 2 * A, &b));
        size_t w = 0;
        const int rc = lanczos_workspace(b, dtype, steps, &w);
        basis_free(b);
        HM_TRY(rc);
        *bytes = std::max(*bytes, w);
    }
    return HM_OK;
}

extern "C" int sector_ground_energies(int n_sites, int two_s, int n_bonds, const int32_t *u, const int32_t *v,
                                      const double *J, int steps, uint64_t seed, int dtype, void *work,
                                      size_t work_bytes, double *e0, int *steps_done, void *stream) {
    if (!e0) return fail(HM_EINVAL, "e0 is NULL");
    if (n_sites < 1 || two_s < 1) return fail(HM_EINVAL, "n_sites and two_s must be positive");
    HM_TRY(bonds_check(n_sites, n_bonds, u, v, J));
    const int nsec = two_s * n_sites + 1;
    std::vector<double> al((size_t)std::max(steps, 1)), be((size_t)std::max(steps, 1));
    for (int A = 0; A < nsec; ++A) {
        hm_basis *b = nullptr;
        HM_TRY(basis_build(n_sites, two_s, two_s * n_sites - 2 * A, &b));
        int done = 0;
        double rz = 0.0;
        int rc = lanczos_run(b, n_bonds, u, v, J, nullptr, sector_seed(seed, A), steps, dtype, work, work_bytes,
                             al.data(), be.data(), &done, &rz, 1, stream);
        basis_free(b);
        if (rc < 0) return rc;
        e0[A] = rz;
        if (steps_done) steps_done[A] = done;
    }
    return HM_OK;
}
