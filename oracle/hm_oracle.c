/*
 * hm_oracle.c -- TEST INFRASTRUCTURE, not part of the product path.
 *
 * A plain, slow, obviously correct CPU restatement of the sector Lanczos method of
 * Schnack, Hage and Schmidt, "Optimized implementation of the Lanczos method for
 * magnetic systems" (J. Comput. Phys.; arXiv:0706.3293):
 *   - the isotropic Heisenberg model, Eq. (E-2-1), with digits a = s - m (Sec. 2);
 *   - the subspace dimension table D(N, A), Eq. (E-3-c) (Sec. 3);
 *   - the direct index -> state decoding (Sec. 3.1), the successor rule (Sec. 3.1)
 *     and the state -> index encoding (Sec. 3.2);
 *   - the row-oriented matrix-vector product, Eq. (E-4-b) (Sec. 4), with the row loop
 *     parallelised over host threads exactly as the paper does with openMP;
 *   - a plain three-term Lanczos recurrence and a Sturm-bisection eigensolver for the
 *     tridiagonal matrix (the Lanczos method the paper builds on, Sec. 1 and 4).
 *
 * Only tests/, __graft_entry__.smoke() and bench.py's CPU legs load this library.  It
 * shares no code, header, table or helper with the CUDA library; the two meet only in
 * the seeded input generators (SplitMix64, implemented independently on each side).
 *
 * Conventions (the readings of the paper this file fixes):
 *   - positions are 0-based in memory: dig[k-1] holds the paper's a_k, k = 1..N;
 *   - indices are 0-based: paper index i corresponds to i - 1 here;
 *   - position N is the most significant digit of the ordering (Eq. E-3-a: a_1 varies
 *     fastest);
 *   - every bond (u, v) of the list is one term -J s_u.s_v of Eq. (E-2-1) (ordered
 *     pairs are not doubled); u == v is rejected by the callers.
 */
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#include <math.h>
#include <float.h>
#ifdef _OPENMP
#include <omp.h>
#endif

typedef struct {
    int N;          /* number of spins */
    int S2;         /* 2s; each digit a_k runs over 0..S2 */
    int A;          /* sector: digit sum A = N s - M */
    int W;          /* row length of the D table: S2*N + 1 */
    int64_t dim;    /* D(N, A) */
    int64_t *D;     /* D(k, a), k = 0..N, a = 0..S2*N, row-major */
} orc_basis;

/* D(k, a) with the convention of Sec. 3: zero whenever a is outside 0..2sk. */
static int64_t orc_D(const orc_basis *b, int k, int a)
{
    if (k < 0 || k > b->N || a < 0 || a > b->S2 * k) return 0;
    return b->D[(int64_t)k * b->W + a];
}

int64_t orc_table(const orc_basis *b, int k, int a) { return orc_D(b, k, a); }

/* Builds D by the recursion of Eq. (E-3-c):
 *   D(0, 0) = 1,  D(k, a) = sum_{n=0}^{2s} D(k-1, a-n).
 * Returns NULL on bad arguments or when a table entry overflows int64. */
orc_basis *orc_basis_new(int N, int S2, int A)
{
    if (N < 1 || N > 64 || S2 < 1 || S2 > 16 || A < 0 || A > S2 * N) return NULL;
    orc_basis *b = (orc_basis *)calloc(1, sizeof(orc_basis));
    if (!b) return NULL;
    b->N = N; b->S2 = S2; b->A = A; b->W = S2 * N + 1;
    b->D = (int64_t *)calloc((size_t)(N + 1) * b->W, sizeof(int64_t));
    if (!b->D) { free(b); return NULL; }
    b->D[0] = 1;
    for (int k = 1; k <= N; ++k) {
        for (int a = 0; a <= S2 * k; ++a) {
            int64_t sum = 0;
            for (int n = 0; n <= S2; ++n) {
                int64_t t = orc_D(b, k - 1, a - n);
                if (__builtin_add_overflow(sum, t, &sum)) { free(b->D); free(b); return NULL; }
            }
            b->D[(int64_t)k * b->W + a] = sum;
        }
    }
    b->dim = orc_D(b, N, A);
    return b;
}

void orc_basis_free(orc_basis *b) { if (b) { free(b->D); free(b); } }
int64_t orc_basis_dim(const orc_basis *b) { return b->dim; }

/* The order of the basis (Eq. E-3-a): |a_1 .. a_N> runs through the digit strings like
 * the numbers sum_k a_k (2s+1)^(k-1), position N most significant, keeping those with
 * digit sum A; the index of a state is the number of sector states before it.
 *
 * Counting them (state -> index, the map Sec. 3.2 computes): a sector state b comes
 * before a exactly when, at the highest position k where the two differ, b_k < a_k.  For
 * a fixed k and a fixed smaller digit n there, the positions above k copy a and the k-1
 * positions below carry the rest of the digit sum, A - n - (a_{k+1} + .. + a_N), in any
 * arrangement: D(k-1, that rest) states by the definition of D (Eq. E-3-c).  Hence
 *     index(a) = sum_{k=1..N} sum_{n < a_k} D(k-1, A - n - T_k),  T_k = a_{k+1} + .. + a_N,
 * with D zero outside its range.  Returns -1 when the digits are not in the sector. */
int64_t orc_encode(const orc_basis *b, const int32_t *dig)
{
    int total = 0;
    for (int k = 0; k < b->N; ++k) {
        if (dig[k] < 0 || dig[k] > b->S2) return -1;
        total += dig[k];
    }
    if (total != b->A) return -1;
    /* suffix[k] = T_k = a_{k+1} + .. + a_N (suffix[N] = 0) */
    int suffix[65];
    suffix[b->N] = 0;
    for (int k = b->N; k >= 1; --k) suffix[k - 1] = suffix[k] + dig[k - 1];
    int64_t count = 0;
    for (int k = 1; k <= b->N; ++k)
        for (int n = 0; n < dig[k - 1]; ++n) count += orc_D(b, k - 1, b->A - n - suffix[k]);
    return count;
}

/* Index -> state (Sec. 3.1), by inverting that count from the top.  Once the digits
 * above position k are fixed (digit sum T_k), the states sharing them are consecutive in
 * the order, and among them those with digit n at position k come before those with a
 * larger digit there; the ones with digit m number D(k-1, A - m - T_k).  So the digit at
 * position k is the n whose run of states holds the rank r left over from the positions
 * above: the last n with P(n) = sum_{m < n} D(k-1, A - m - T_k) <= r; r then drops by P(n).
 * Position 1 takes whatever digit sum is left.  Returns 0, or -1 for an index outside the
 * sector. */
int orc_decode(const orc_basis *b, int64_t i, int32_t *dig)
{
    if (i < 0 || i >= b->dim) return -1;
    int64_t r = i;
    int Tk = 0;                              /* digit sum of the positions above k */
    for (int k = b->N; k >= 2; --k) {
        int64_t P = 0;                       /* states before the run of digit n */
        int n = 0;
        while (n < b->S2) {
            const int64_t next = P + orc_D(b, k - 1, b->A - n - Tk);
            if (next > r) break;             /* rank r lies in the run of digit n */
            P = next;
            ++n;
        }
        if (r - P >= orc_D(b, k - 1, b->A - n - Tk)) return -1;
        dig[k - 1] = n;
        r -= P;
        Tk += n;
    }
    dig[0] = b->A - Tk;
    if (dig[0] < 0 || dig[0] > b->S2 || r != 0) return -1;
    return 0;
}

/* Sec. 3.1, the successor in lexicographic order ("balls in boxes"):
 *   1. find the leftmost box k that is not empty and whose right neighbour holds
 *      fewer than 2s balls (none: the state is the last one);
 *   2. move one ball from box k to box k+1;
 *   3. take all balls out of boxes 1..k and refill them from the left, 2s per box.
 * Returns 1 if a successor exists (dig is overwritten), else 0. */
int orc_successor(int N, int S2, int32_t *dig)
{
    int k = -1;
    for (int p = 0; p + 1 < N; ++p)
        if (dig[p] > 0 && dig[p + 1] < S2) { k = p; break; }
    if (k < 0) return 0;
    dig[k] -= 1;
    dig[k + 1] += 1;
    int balls = 0;
    for (int p = 0; p <= k; ++p) { balls += dig[p]; dig[p] = 0; }
    for (int p = 0; p <= k && balls > 0; ++p) {
        int t = balls < S2 ? balls : S2;
        dig[p] = t;
        balls -= t;
    }
    return 1;
}

/* ---- the bond term s_u . s_v = s^z_u s^z_v + 1/2 (s+_u s-_v + s-_u s+_v) (Eq. E-2-1) ----
 * With a = s - m: s^z |a> = (s - a)|a>, s+ lowers the digit, s- raises it:
 *   s+ |a> = sqrt(a (2s - a + 1)) |a - 1>,   s- |a> = sqrt((2s - a)(a + 1)) |a + 1>.
 * The exchange element is 1/2 * sqrt(product of the two radicands), the square root of
 * an integer, correctly rounded by IEEE sqrt. */
static double orc_mz(int S2, int a) { return 0.5 * (double)S2 - (double)a; }

static int64_t orc_rad_up(int S2, int a) { return (int64_t)a * (S2 - a + 1); }   /* for s+ */
static int64_t orc_rad_dn(int S2, int a) { return (int64_t)(S2 - a) * (a + 1); } /* for s- */

/* y_i for one row: applies every bond to the row's own state |i> (the final state of
 * Eq. E-4-b), which yields the initial states j(i) with their matrix elements, and sums
 * <i|H|j> x_j.  H = -sum_b J_b s_u . s_v.  'nnz' (optional) counts the non-zero
 * elements of the row: one diagonal plus every allowed exchange. */
static double orc_row(const orc_basis *b, int nb, const int32_t *u, const int32_t *v,
                      const double *J, const double *x, int64_t i, int32_t *dig,
                      int64_t *nnz)
{
    const int S2 = b->S2;
    orc_decode(b, i, dig);
    double diag = 0.0, off = 0.0;
    int64_t cnt = 1;
    for (int t = 0; t < nb; ++t) {
        int p = u[t], q = v[t];
        int ap = dig[p], aq = dig[q];
        diag += -J[t] * orc_mz(S2, ap) * orc_mz(S2, aq);
        if (ap >= 1 && aq <= S2 - 1) {             /* 1/2 s+_u s-_v */
            double c = 0.5 * sqrt((double)(orc_rad_up(S2, ap) * orc_rad_dn(S2, aq)));
            dig[p] = ap - 1; dig[q] = aq + 1;
            int64_t j = orc_encode(b, dig);
            dig[p] = ap; dig[q] = aq;
            off += -J[t] * c * x[j];
            ++cnt;
        }
        if (ap <= S2 - 1 && aq >= 1) {             /* 1/2 s-_u s+_v */
            double c = 0.5 * sqrt((double)(orc_rad_dn(S2, ap) * orc_rad_up(S2, aq)));
            dig[p] = ap + 1; dig[q] = aq - 1;
            int64_t j = orc_encode(b, dig);
            dig[p] = ap; dig[q] = aq;
            off += -J[t] * c * x[j];
            ++cnt;
        }
    }
    if (nnz) *nnz = cnt;
    return diag * x[i] + off;
}

static int orc_bonds_ok(const orc_basis *b, int nb, const int32_t *u, const int32_t *v)
{
    if (nb < 0) return 0;
    for (int t = 0; t < nb; ++t)
        if (u[t] < 0 || u[t] >= b->N || v[t] < 0 || v[t] >= b->N || u[t] == v[t]) return 0;
    return 1;
}

/* Eq. (E-4-b): y = H x over the rows [r0, r1), the row index being the outer (parallel)
 * loop; rows never write each other's output.  Returns 0 or -1 on bad bonds/range. */
int orc_matvec_rows(const orc_basis *b, int nb, const int32_t *u, const int32_t *v,
                    const double *J, const double *x, double *y, int64_t r0, int64_t r1)
{
    if (!orc_bonds_ok(b, nb, u, v) || r0 < 0 || r1 > b->dim || r0 > r1) return -1;
    #pragma omp parallel
    {
        int32_t dig[64];
        #pragma omp for schedule(dynamic, 4096)
        for (int64_t i = r0; i < r1; ++i)
            y[i - r0] = orc_row(b, nb, u, v, J, x, i, dig, NULL);
    }
    return 0;
}

int orc_matvec(const orc_basis *b, int nb, const int32_t *u, const int32_t *v,
               const double *J, const double *x, double *y)
{
    return orc_matvec_rows(b, nb, u, v, J, x, y, 0, b->dim);
}

/* Number of non-zero matrix elements in rows [r0, r1) (diagonal counted once per row). */
int64_t orc_count_nnz(const orc_basis *b, int nb, const int32_t *u, const int32_t *v,
                      int64_t r0, int64_t r1)
{
    if (!orc_bonds_ok(b, nb, u, v) || r0 < 0 || r1 > b->dim || r0 > r1) return -1;
    int64_t total = 0;
    #pragma omp parallel reduction(+:total)
    {
        int32_t dig[64];
        #pragma omp for schedule(dynamic, 4096)
        for (int64_t i = r0; i < r1; ++i) {
            const int S2 = b->S2;
            orc_decode(b, i, dig);
            int64_t cnt = 1;
            for (int t = 0; t < nb; ++t) {
                int ap = dig[u[t]], aq = dig[v[t]];
                if (ap >= 1 && aq <= S2 - 1) ++cnt;
                if (ap <= S2 - 1 && aq >= 1) ++cnt;
            }
            total += cnt;
        }
    }
    return total;
}

/* out[t] = sum_i g_i [(s_u . s_v) x]_i for every bond t (no coupling, no sign).  Because
 * H is linear in the couplings, d(g^T H x)/dJ_t = -out[t]. */
int orc_bond_corr(const orc_basis *b, int nb, const int32_t *u, const int32_t *v,
                  const double *g, const double *x, double *out)
{
    if (!orc_bonds_ok(b, nb, u, v)) return -1;
    for (int t = 0; t < nb; ++t) out[t] = 0.0;
    #pragma omp parallel
    {
        int32_t dig[64];
        double *acc = (double *)calloc(nb > 0 ? nb : 1, sizeof(double));
        #pragma omp for schedule(static)
        for (int64_t i = 0; i < b->dim; ++i) {
            const int S2 = b->S2;
            orc_decode(b, i, dig);
            for (int t = 0; t < nb; ++t) {
                int p = u[t], q = v[t];
                int ap = dig[p], aq = dig[q];
                double r = orc_mz(S2, ap) * orc_mz(S2, aq) * x[i];
                if (ap >= 1 && aq <= S2 - 1) {
                    double c = 0.5 * sqrt((double)(orc_rad_up(S2, ap) * orc_rad_dn(S2, aq)));
                    dig[p] = ap - 1; dig[q] = aq + 1;
                    r += c * x[orc_encode(b, dig)];
                    dig[p] = ap; dig[q] = aq;
                }
                if (ap <= S2 - 1 && aq >= 1) {
                    double c = 0.5 * sqrt((double)(orc_rad_dn(S2, ap) * orc_rad_up(S2, aq)));
                    dig[p] = ap + 1; dig[q] = aq - 1;
                    r += c * x[orc_encode(b, dig)];
                    dig[p] = ap; dig[q] = aq;
                }
                acc[t] += g[i] * r;
            }
        }
        #pragma omp critical
        for (int t = 0; t < nb; ++t) out[t] += acc[t];
        free(acc);
    }
    return 0;
}

/* ---- plain Lanczos recurrence (the method of Sec. 1/4, reference [Lanczos 1950]) ----
 * v_1 = v0/|v0|, beta_0 = 0, then for j = 1..steps:
 *   u = H v_j - beta_{j-1} v_{j-1},  alpha_j = v_j . u,  w = u - alpha_j v_j,
 *   beta_j = |w|,  v_{j+1} = w / beta_j.
 * No re-orthogonalisation.  The run stops after step j (breakdown) when
 * beta_j <= tol * max(|alpha_1..alpha_j|, beta_1..beta_{j-1}).
 * If coef is given, psi accumulates sum_j coef[j] v_j (the Ritz vector of a second pass).
 * Returns the number of steps done (>= 1), or -1 on error. */
int orc_lanczos(const orc_basis *b, int nb, const int32_t *u, const int32_t *v,
                const double *J, const double *v0, int steps, double tol,
                double *alpha, double *beta, const double *coef, double *psi)
{
    if (!orc_bonds_ok(b, nb, u, v) || steps < 1) return -1;
    const int64_t n = b->dim;
    double *vp = (double *)calloc(n, sizeof(double));
    double *vc = (double *)malloc(n * sizeof(double));
    double *w = (double *)malloc(n * sizeof(double));
    if (!vp || !vc || !w) { free(vp); free(vc); free(w); return -1; }
    double nrm = 0.0;
    for (int64_t i = 0; i < n; ++i) nrm += v0[i] * v0[i];
    nrm = sqrt(nrm);
    for (int64_t i = 0; i < n; ++i) vc[i] = v0[i] / nrm;
    if (psi) for (int64_t i = 0; i < n; ++i) psi[i] = 0.0;
    double bprev = 0.0, scale = 0.0;
    int done = 0;
    for (int j = 0; j < steps; ++j) {
        if (psi) for (int64_t i = 0; i < n; ++i) psi[i] += coef[j] * vc[i];
        orc_matvec(b, nb, u, v, J, vc, w);
        for (int64_t i = 0; i < n; ++i) w[i] -= bprev * vp[i];
        double a = 0.0;
        for (int64_t i = 0; i < n; ++i) a += vc[i] * w[i];
        for (int64_t i = 0; i < n; ++i) w[i] -= a * vc[i];
        double bb = 0.0;
        for (int64_t i = 0; i < n; ++i) bb += w[i] * w[i];
        bb = sqrt(bb);
        alpha[j] = a;
        beta[j] = bb;
        done = j + 1;
        if (fabs(a) > scale) scale = fabs(a);
        if (bb <= tol * scale) break;
        if (bb > scale) scale = bb;
        for (int64_t i = 0; i < n; ++i) { vp[i] = vc[i]; vc[i] = w[i] / bb; }
        bprev = bb;
    }
    free(vp); free(vc); free(w);
    return done;
}

/* Number of eigenvalues of the symmetric tridiagonal T (diagonal al[0..m-1],
 * off-diagonal be[0..m-2]) below x, from the signs of the Sturm sequence
 * q_1 = al_1 - x, q_i = al_i - x - be_{i-1}^2 / q_{i-1} (a zero pivot is replaced by
 * -pivmin). */
static int orc_sturm(int m, const double *al, const double *be, double x, double pivmin)
{
    int c = 0;
    double q = al[0] - x;
    if (fabs(q) < pivmin) q = -pivmin;
    if (q < 0) ++c;
    for (int i = 1; i < m; ++i) {
        q = al[i] - x - be[i - 1] * be[i - 1] / q;
        if (fabs(q) < pivmin) q = -pivmin;
        if (q < 0) ++c;
    }
    return c;
}

/* The k lowest eigenvalues of T by bisection on the Sturm count, starting from the
 * Gershgorin interval, until the bracket cannot shrink further. */
void orc_tridiag_lowest(int m, const double *al, const double *be, int k, double *out)
{
    double lo = DBL_MAX, hi = -DBL_MAX, bmax = 0.0;
    for (int i = 0; i < m; ++i) {
        double r = (i > 0 ? fabs(be[i - 1]) : 0.0) + (i < m - 1 ? fabs(be[i]) : 0.0);
        if (al[i] - r < lo) lo = al[i] - r;
        if (al[i] + r > hi) hi = al[i] + r;
        if (i < m - 1 && fabs(be[i]) > bmax) bmax = fabs(be[i]);
    }
    double pivmin = DBL_MIN * (bmax * bmax > 1.0 ? bmax * bmax : 1.0);
    double pad = 2.0 * DBL_EPSILON * (fabs(lo) > fabs(hi) ? fabs(lo) : fabs(hi)) + pivmin;
    lo -= pad; hi += pad;
    for (int e = 1; e <= k && e <= m; ++e) {
        double a = lo, c = hi;
        for (int it = 0; it < 400; ++it) {
            double mid = 0.5 * (a + c);
            if (mid <= a || mid >= c) break;
            if (orc_sturm(m, al, be, mid, pivmin) >= e) c = mid; else a = mid;
        }
        out[e - 1] = 0.5 * (a + c);
    }
}

/* ---- SplitMix64 (Steele, Lea, Flood, OOPSLA 2014): the seeded start vectors ----
 * Output number t (0-based) of the generator seeded with s is mix(s + (t + 1) * gamma). */
static const uint64_t ORC_GAMMA = 0x9E3779B97F4A7C15ULL;

static uint64_t orc_mix64(uint64_t z)
{
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ULL;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBULL;
    return z ^ (z >> 31);
}

uint64_t orc_splitmix(uint64_t seed, uint64_t t) { return orc_mix64(seed + (t + 1) * ORC_GAMMA); }

/* x_t = 2 u_t - 1 with u_t = (out_t >> 11) * 2^-53, uniform on [-1, 1). */
void orc_start_uniform(uint64_t seed, int64_t n, double *out)
{
    #pragma omp parallel for schedule(static)
    for (int64_t t = 0; t < n; ++t)
        out[t] = 2.0 * ((double)(orc_splitmix(seed, (uint64_t)t) >> 11) * 0x1.0p-53) - 1.0;
}

/* x_t = -1 if the top bit of out_t is set, else +1. */
void orc_start_pm1(uint64_t seed, int64_t n, double *out)
{
    #pragma omp parallel for schedule(static)
    for (int64_t t = 0; t < n; ++t)
        out[t] = (orc_splitmix(seed, (uint64_t)t) >> 63) ? -1.0 : 1.0;
}

/* Seed of the start vector of (sector A, vector r) in a batched run. */
uint64_t orc_stream_seed(uint64_t seed, int A, int r)
{
    return orc_splitmix(seed, ((uint64_t)A << 20) + (uint64_t)r);
}

int orc_num_threads(void)
{
#ifdef _OPENMP
    return omp_get_max_threads();
#else
    return 1;
#endif
}
