// momentum.cu -- translation symmetry of a ring: the momentum blocks k = 0 and k = pi of a
// magnetisation sector.  The paper names further symmetries as a way to shrink H(M)
// beyond the M sectors; the construction here is the textbook one for the cyclic group of
// the ring (T: site u -> u + 1 mod N), restricted to the two real characters
// chi(n) = 1 (k = 0) and chi(n) = (-1)^n (k = pi, even N).
//
// Basis: one state per orbit of T inside the sector, its representative r the orbit member
// with the smallest packed digit word; with p the orbit's period (T^p r = r),
//     |r^> = p^(-1/2) sum_{m < p} chi(m) T^m |r>,
// present when chi(p) = 1 (every orbit for k = 0, even periods for k = pi).  For a term
// h |s> of H|r> with s = T^l r' (r' the representative of s's orbit),
//     H |r^> = sum over terms h chi(l) sqrt(p_r / p_r') |r'^>,
// and H is real symmetric on these states, so row r of y = H x is the same sum over the
// terms of H|r> applied to x_{r'}.
//
// GB300 form: a table over the whole sector, filled once, maps every sector index (the
// paper's coding, Sec. 3) to (representative number, shift l, period): a row decodes its
// representative, applies the bond terms, encodes each target with the sector codec and
// reads the table there -- one gather replaces the orbit search of every target.  The
// table takes 8 bytes per sector state (4.8 GB at N = 32), small next to the 280 GB HBM.
#include <algorithm>
#include <cmath>
#include <vector>

#include "ef64.cuh"
#include "hm_row.cuh"

namespace hm {

constexpr int MOM_NT = 256;
constexpr int MOM_PER = 32;          // consecutive sector indices a thread ranks
constexpr int MOM_CH = MOM_NT * MOM_PER;
constexpr uint64_t MOM_NONE = ~0ull;

struct MomOrbit {
    uint64_t rep;                    // smallest packed word of the orbit
    int shift;                       // l with T^l rep = w
    int period;                      // smallest p > 0 with T^p w = w
};

// one translation u -> u + 1 of a packed digit word of N digits
__device__ __forceinline__ uint64_t mom_rot(uint64_t w, int N, int bits, uint64_t mask) {
    return ((w << bits) | (w >> ((N - 1) * bits))) & mask;
}

__device__ __forceinline__ MomOrbit mom_orbit(uint64_t w, int N, int bits) {
    const uint64_t mask = N * bits >= 64 ? ~0ull : ((1ull << (N * bits)) - 1ull);
    MomOrbit o{w, 0, N};
    uint64_t t = w;
    int nmin = 0;
    for (int n = 1; n < N; ++n) {
        t = mom_rot(t, N, bits, mask);
        if (t == w && o.period == N) o.period = n;
        if (t < o.rep) { o.rep = t; nmin = n; }
    }
    o.shift = (N - nmin) % N;        // T^nmin w = rep, so w = T^(N - nmin) rep
    return o;
}

// chi(p) = 1: the orbit contributes a basis state
__device__ __forceinline__ bool mom_ok(int period, int kpi) { return !kpi || (period & 1) == 0; }

// chunk c of the sector: number of representatives of compatible orbits
__global__ void __launch_bounds__(MOM_NT) k_mom_count(SectorView sv, int kpi, uint32_t *__restrict__ counts) {
    __shared__ uint32_t cd[4096];
    __shared__ int red[MOM_NT / 32];
    for (int k = threadIdx.x; k < sv.cd_len; k += MOM_NT) cd[k] = ((const uint32_t *)sv.cd)[k];
    __syncthreads();
    Codec<uint32_t> c{cd, sv.N, sv.S2, sv.A, sv.bits, sv.cd_w, sv.cd_rowlen};
    const uint64_t i0 = (uint64_t)blockIdx.x * MOM_CH + (uint64_t)threadIdx.x * MOM_PER;
    int n = 0;
    for (int j = 0; j < MOM_PER; ++j) {
        const uint64_t i = i0 + j;
        if (i >= sv.dim) break;
        const uint64_t w = c.decode((uint32_t)i);
        const MomOrbit o = mom_orbit(w, sv.N, sv.bits);
        n += (o.rep == w && mom_ok(o.period, kpi)) ? 1 : 0;
    }
    for (int o = 16; o > 0; o >>= 1) n += __shfl_down_sync(0xffffffffu, n, o);
    if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = n;
    __syncthreads();
    if (threadIdx.x == 0) {
        int t = 0;
        for (int k = 0; k < MOM_NT / 32; ++k) t += red[k];
        counts[blockIdx.x] = (uint32_t)t;
    }
}

// representatives of chunk c numbered in index order from off[c]: reps[number] = sector
// index, map[index] = number | period << 40 (shift 0)
__global__ void __launch_bounds__(MOM_NT) k_mom_reps(SectorView sv, int kpi, const uint32_t *__restrict__ off,
                                                      uint32_t *__restrict__ reps, uint64_t *__restrict__ map) {
    __shared__ uint32_t cd[4096];
    __shared__ int tcount[MOM_NT];
    for (int k = threadIdx.x; k < sv.cd_len; k += MOM_NT) cd[k] = ((const uint32_t *)sv.cd)[k];
    __syncthreads();
    Codec<uint32_t> c{cd, sv.N, sv.S2, sv.A, sv.bits, sv.cd_w, sv.cd_rowlen};
    const uint64_t i0 = (uint64_t)blockIdx.x * MOM_CH + (uint64_t)threadIdx.x * MOM_PER;
    uint32_t flags = 0;
    uint8_t per[MOM_PER];
    for (int j = 0; j < MOM_PER; ++j) {
        const uint64_t i = i0 + j;
        per[j] = 0;
        if (i >= sv.dim) continue;
        const uint64_t w = c.decode((uint32_t)i);
        const MomOrbit o = mom_orbit(w, sv.N, sv.bits);
        if (o.rep == w && mom_ok(o.period, kpi)) {
            flags |= 1u << j;
            per[j] = (uint8_t)o.period;
        }
    }
    tcount[threadIdx.x] = __popc(flags);
    __syncthreads();
    if (threadIdx.x == 0) {          // exclusive scan of the thread counts, in thread order
        int s = 0;
        for (int k = 0; k < MOM_NT; ++k) {
            const int t = tcount[k];
            tcount[k] = s;
            s += t;
        }
    }
    __syncthreads();
    uint32_t num = off[blockIdx.x] + (uint32_t)tcount[threadIdx.x];
    for (int j = 0; j < MOM_PER; ++j)
        if (flags & (1u << j)) {
            reps[num] = (uint32_t)(i0 + j);
            map[i0 + j] = (uint64_t)num | ((uint64_t)per[j] << 40);
            ++num;
        }
}

// every other sector index: its representative's number, the shift and the period, or
// MOM_NONE for orbits without a basis state
__global__ void __launch_bounds__(MOM_NT) k_mom_map(SectorView sv, int kpi, uint64_t *__restrict__ map) {
    __shared__ uint32_t cd[4096];
    for (int k = threadIdx.x; k < sv.cd_len; k += MOM_NT) cd[k] = ((const uint32_t *)sv.cd)[k];
    __syncthreads();
    Codec<uint32_t> c{cd, sv.N, sv.S2, sv.A, sv.bits, sv.cd_w, sv.cd_rowlen};
    for (uint64_t i = (uint64_t)blockIdx.x * MOM_NT + threadIdx.x; i < sv.dim; i += (uint64_t)gridDim.x * MOM_NT) {
        const uint64_t w = c.decode((uint32_t)i);
        const MomOrbit o = mom_orbit(w, sv.N, sv.bits);
        if (!mom_ok(o.period, kpi)) {
            map[i] = MOM_NONE;
        } else if (o.rep != w) {
            const uint64_t e = map[c.encode(o.rep)];      // written by k_mom_reps
            map[i] = (e & 0xFFFFFFFFull) | ((uint64_t)o.shift << 32) | ((uint64_t)o.period << 40);
        }
    }
}

// y = H x on the momentum basis (sums in binary64, T = double or float).  A target's
// sector index is the row's own index plus the rank change of positions p..q (Sec. 3.2,
// Codec::delta), so nearest- and next-nearest-neighbour exchanges cost two or three table
// reads instead of a full encode; the factor sqrt(p_r) is applied once per row.
template <class T>
__global__ void __launch_bounds__(MOM_NT) k_mom_matvec(SectorView sv, BondParams bp, int kpi, uint64_t nrep,
                                                        const uint32_t *__restrict__ reps,
                                                        const uint64_t *__restrict__ map, const T *__restrict__ x,
                                                        T *__restrict__ y) {
    __shared__ uint32_t cd[4096];
    __shared__ double sq[65], isq[65];   // sqrt(p), 1 / sqrt(p), p = 0..64
    // per bond -J_b / 4 and -J_b / 2: the diagonal term is jq (2s - 2a_p)(2s - 2a_q) and
    // the s = 1/2 exchange coefficient jh (few binary64 operations per bond: this GPU's
    // FP64 pipe bounded the first version at 82 %)
    __shared__ double jq[HM_MAX_BONDS], jh[HM_MAX_BONDS];
    for (int k = threadIdx.x; k < sv.cd_len; k += MOM_NT) cd[k] = ((const uint32_t *)sv.cd)[k];
    for (int k = threadIdx.x; k <= 64; k += MOM_NT) {
        sq[k] = sqrt((double)k);
        isq[k] = k ? 1.0 / sqrt((double)k) : 0.0;
    }
    __shared__ double jqsum;
    for (int k = threadIdx.x; k < bp.nb; k += MOM_NT) {
        jq[k] = 0.25 * bp.jm[k];
        jh[k] = 0.5 * bp.jm[k];
    }
    if (threadIdx.x == 0) {
        double t = 0.0;
        for (int k = 0; k < bp.nb; ++k) t += 0.25 * bp.jm[k];
        jqsum = t;
    }
    __syncthreads();
    Codec<uint32_t> c{cd, sv.N, sv.S2, sv.A, sv.bits, sv.cd_w, sv.cd_rowlen};
    for (uint64_t r = (uint64_t)blockIdx.x * MOM_NT + threadIdx.x; r < nrep; r += (uint64_t)gridDim.x * MOM_NT) {
        const uint32_t i = reps[r];
        const uint64_t w = c.decode(i);
        if (sv.S2 == 1) {
            // s = 1/2: a bond's exchange is allowed exactly when its spins differ, and then
            // its diagonal term is -jq instead of +jq: dg = sum jq - 2 sum over those bonds of
            // jq.  Targets of full period N share the factor 1 / sqrt(N).
            double sd = 0.0, accn = 0.0, acco = 0.0;
            for (int b = 0; b < bp.nb; ++b) {
                const int p = bp.p[b], q = bp.q[b];
                const int ap = dig(w, p, 1), aq = dig(w, q, 1);
                if (ap == aq) continue;
                sd += jq[b];
                const uint64_t e = map[i + c.delta(w, p, q, ap ? -1 : 1)];
                if (e == MOM_NONE) continue;
                const double f = (kpi && ((e >> 32) & 1)) ? -jh[b] : jh[b];
                const int per = (int)((e >> 40) & 0xFF);
                if (per == sv.N) accn = fma(f, (double)x[(uint32_t)e], accn);
                else acco = fma(f * isq[per], (double)x[(uint32_t)e], acco);
            }
            const double dg = jqsum - 2.0 * sd;
            y[r] = (T)(dg * (double)x[r] + sq[(map[i] >> 40) & 0xFF] * (isq[sv.N] * accn + acco));
            continue;
        }
        double dg = 0.0, acc = 0.0;
        for (int b = 0; b < bp.nb; ++b) {
            const int p = bp.p[b], q = bp.q[b];
            const int ap = dig(w, p, sv.bits), aq = dig(w, q, sv.bits);
            dg = fma((double)((sv.S2 - 2 * ap) * (sv.S2 - 2 * aq)), jq[b], dg);
            // s+_p s-_q (a_p - 1, a_q + 1) and s-_p s+_q (a_p + 1, a_q - 1), Eq. E-2-1
            for (int d = 0; d < 2; ++d) {
                const bool ok = d == 0 ? (ap >= 1 && aq < sv.S2) : (ap < sv.S2 && aq >= 1);
                if (!ok) continue;
                const uint64_t e = map[i + c.delta(w, p, q, d == 0 ? -1 : 1)];
                if (e == MOM_NONE) continue;
                const double f = bp.jm[b] * (d == 0 ? bp.hs_pdn[ap * 8 + aq] : bp.hs_pup[ap * 8 + aq]);
                const double v = f * isq[(e >> 40) & 0xFF] * (double)x[(uint32_t)e];
                acc += (kpi && ((e >> 32) & 1)) ? -v : v;
            }
        }
        y[r] = (T)(dg * (double)x[r] + sq[(map[i] >> 40) & 0xFF] * acc);
    }
}

// terms of the product: per representative 1 (the diagonal) + its allowed exchanges whose
// target orbit has a basis state; summed into *out
__global__ void __launch_bounds__(MOM_NT) k_mom_count_nnz(SectorView sv, BondParams bp, uint64_t nrep,
                                                           const uint32_t *__restrict__ reps,
                                                           const uint64_t *__restrict__ map,
                                                           unsigned long long *out) {
    __shared__ uint32_t cd[4096];
    __shared__ unsigned long long red[MOM_NT / 32];
    for (int k = threadIdx.x; k < sv.cd_len; k += MOM_NT) cd[k] = ((const uint32_t *)sv.cd)[k];
    __syncthreads();
    Codec<uint32_t> c{cd, sv.N, sv.S2, sv.A, sv.bits, sv.cd_w, sv.cd_rowlen};
    unsigned long long n = 0;
    for (uint64_t r = (uint64_t)blockIdx.x * MOM_NT + threadIdx.x; r < nrep; r += (uint64_t)gridDim.x * MOM_NT) {
        const uint64_t w = c.decode(reps[r]);
        n += 1;
        for (int b = 0; b < bp.nb; ++b) {
            const int p = bp.p[b], q = bp.q[b];
            const int ap = dig(w, p, sv.bits), aq = dig(w, q, sv.bits);
            const uint64_t up = (uint64_t)1 << (p * sv.bits), uq = (uint64_t)1 << (q * sv.bits);
            if (ap >= 1 && aq < sv.S2 && map[c.encode(w - up + uq)] != MOM_NONE) ++n;   // full encode: an
            if (ap < sv.S2 && aq >= 1 && map[c.encode(w + up - uq)] != MOM_NONE) ++n;   // independent count
        }
    }
    for (int o = 16; o > 0; o >>= 1) n += __shfl_down_sync(0xffffffffu, n, o);
    if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = n;
    __syncthreads();
    if (threadIdx.x == 0) {
        unsigned long long t = 0;
        for (int k = 0; k < MOM_NT / 32; ++k) t += red[k];
        atomicAdd(out, t);
    }
}

// ---- host -----------------------------------------------------------------------------------

int mom_count_nnz(const hm_basis *b, const BondParams &bp, int64_t *nnz, cudaStream_t st) {
    HM_CUDA(cudaMemsetAsync(nnz, 0, sizeof(int64_t), st));
    k_mom_count_nnz<<<grid_blocks(b->view.dim, MOM_NT), MOM_NT, 0, st>>>(
        b->mom_sector, bp, b->view.dim, (const uint32_t *)b->d_mom_reps, (const uint64_t *)b->d_mom_map,
        (unsigned long long *)nnz);
    HM_CUDA(cudaGetLastError());
    return HM_OK;
}

// the bond list must map onto itself under u -> u + 1 (mod N) with equal couplings (summed
// over repeated pairs), so that H commutes with T
int mom_check_bonds(const hm_basis *b, int n_bonds, const int32_t *u, const int32_t *v, const double *J) {
    const int N = b->view.N;
    std::vector<double> Jp((size_t)N * N, 0.0);
    double jmax = 0.0;
    for (int t = 0; t < n_bonds; ++t) {
        const int a = std::min(u[t], v[t]), c = std::max(u[t], v[t]);
        Jp[(size_t)a * N + c] += J[t];
        jmax = std::max(jmax, std::fabs(J[t]));
    }
    for (int a = 0; a < N; ++a)
        for (int c = a + 1; c < N; ++c) {
            const int a2 = (a + 1) % N, c2 = (c + 1) % N;
            const double j2 = Jp[(size_t)std::min(a2, c2) * N + std::max(a2, c2)];
            if (std::fabs(Jp[(size_t)a * N + c] - j2) > 1e-12 * std::max(1.0, jmax))
                return fail(HM_EINVAL, "momentum basis: the bonds are not invariant under the translation u -> u + 1");
        }
    return HM_OK;
}

int mom_matvec(const hm_basis *b, const BondParams &bp, const void *x, void *y, int dtype, cudaStream_t st) {
    const SectorView &sv = b->mom_sector;
    const int nblk = grid_blocks(b->view.dim, MOM_NT);
    const uint32_t *reps = (const uint32_t *)b->d_mom_reps;
    const uint64_t *map = (const uint64_t *)b->d_mom_map;
    const int kpi = b->mom_k != 0;
    if (dtype == HM_F64)
        k_mom_matvec<double><<<nblk, MOM_NT, 0, st>>>(sv, bp, kpi, b->view.dim, reps, map, (const double *)x,
                                                      (double *)y);
    else
        k_mom_matvec<float><<<nblk, MOM_NT, 0, st>>>(sv, bp, kpi, b->view.dim, reps, map, (const float *)x,
                                                     (float *)y);
    HM_CUDA(cudaGetLastError());
    return HM_OK;
}

}  // namespace hm

using namespace hm;

extern "C" int basis_build_momentum(int n_sites, int two_s, int two_m, int k, hm_basis **out) {
    if (!out) return fail(HM_EINVAL, "out is NULL");
    *out = nullptr;
    if (n_sites < 2 || n_sites > 64) return fail(HM_EINVAL, "n_sites must be in 2..64 (got %d)", n_sites);
    if (k != 0 && !(n_sites % 2 == 0 && k == n_sites / 2))
        return fail(HM_EINVAL, "momentum index k must be 0 or N/2 for even N (got %d)", k);
    hm_basis *b = nullptr;
    HM_TRY(basis_build(n_sites, two_s, two_m, &b));
    const SectorView sv = b->view;
    auto reject = [&](const char *why) {
        basis_free(b);
        return fail(HM_EINVAL, "momentum basis: %s", why);
    };
    if (sv.idx64 || sv.dim >= 0xFFFFFFFFull) return reject("the sector must have fewer than 2^32 states");
    if (sv.N * sv.bits > 64) return reject("N digits must fit a 64-bit word");
    if ((size_t)sv.cd_len > 4096) return reject("rank table too large for the momentum kernels");
    const int kpi = k != 0;
    const uint64_t nch = (sv.dim + MOM_CH - 1) / MOM_CH;
    uint32_t *d_cnt = nullptr;
    cudaError_t e = cudaMalloc(&d_cnt, nch * 4);
    if (e != cudaSuccess) { basis_free(b); return cuda_fail(e, "momentum counts"); }
    int rc = HM_OK;
    std::vector<uint32_t> cnt(nch), off(nch);
    uint64_t nrep = 0;
    do {
        k_mom_count<<<(unsigned)nch, MOM_NT>>>(sv, kpi, d_cnt);
        if ((e = cudaGetLastError()) != cudaSuccess || (e = cudaDeviceSynchronize()) != cudaSuccess) {
            rc = cuda_fail(e, "k_mom_count");
            break;
        }
        if ((e = cudaMemcpy(cnt.data(), d_cnt, nch * 4, cudaMemcpyDeviceToHost)) != cudaSuccess) {
            rc = cuda_fail(e, "momentum counts");
            break;
        }
        for (uint64_t c = 0; c < nch; ++c) {
            off[c] = (uint32_t)nrep;
            nrep += cnt[c];
        }
        if (nrep == 0) { rc = fail(HM_EINVAL, "momentum basis: no state has this momentum"); break; }
        const size_t bmap = (sv.dim * 8 + 255) & ~(size_t)255;
        void *dev = nullptr;
        if ((e = cudaMalloc(&dev, bmap + nrep * 4)) != cudaSuccess) { rc = cuda_fail(e, "momentum tables"); break; }
        b->d_mom = dev;
        b->d_mom_map = dev;
        b->d_mom_reps = (unsigned char *)dev + bmap;
        if ((e = cudaMemcpy(d_cnt, off.data(), nch * 4, cudaMemcpyHostToDevice)) != cudaSuccess) {
            rc = cuda_fail(e, "momentum offsets");
            break;
        }
        k_mom_reps<<<(unsigned)nch, MOM_NT>>>(sv, kpi, d_cnt, (uint32_t *)b->d_mom_reps, (uint64_t *)b->d_mom_map);
        k_mom_map<<<grid_blocks(sv.dim, MOM_NT), MOM_NT>>>(sv, kpi, (uint64_t *)b->d_mom_map);
        if ((e = cudaGetLastError()) != cudaSuccess || (e = cudaDeviceSynchronize()) != cudaSuccess) {
            rc = cuda_fail(e, "momentum map");
            break;
        }
    } while (0);
    cudaFree(d_cnt);
    if (rc != HM_OK) {
        basis_free(b);
        return rc;
    }
    b->mom_k = k;
    b->mom_sector = sv;
    b->view.dim = nrep;              // vectors of this basis: one entry per representative
    *out = b;
    return HM_OK;
}
