/*
 * isg_oracle.c -- plain, slow CPU oracle for the exact Ising degeneracy table g(E,M)
 * and the thermodynamics derived from it.
 *
 * TEST INFRASTRUCTURE. Only the test suite, the package's smoke check and the benchmark's
 * CPU-baseline / reference leg may load this library. It shares no code, header, table or
 * constant with the CUDA path, and the CUDA path never calls it.
 *
 * Source of truth: Peretyatko et al., "Rigorous Calculation of the Partition Function for the
 * Finite Number of Ising Spins" (arXiv:1110.2561).
 *
 * Conventions (the readings of the paper that this file implements):
 *  - Spin i of configuration word s is up (S_i = +1) when bit i of s is 1, down (S_i = -1)
 *    otherwise; the paper counts the "units" of the bit-vectors as up spins (Sec. 3a).
 *  - E(s) = -sum over bonds {i,j} of J_ij S_i S_j. Eq. (1) writes a double sum over sites and
 *    their neighbours with a factor 1/2, so each bond counts once (Sec. 2, Eq. 1). The field
 *    term -h*M is kept apart and enters only the thermodynamics.
 *  - M(s) = sum_i S_i, the spin excess (Sec. 2, Sec. 3a). Sec. 3a words it as N minus twice the
 *    number of up spins, which is -M; the sign is read as M = 2*up - N so that h > 0 favours
 *    M > 0. The table g is symmetric under M -> -M at h = 0 in any case.
 *  - Couplings listed more than once for the same unordered pair are summed; a pair whose
 *    summed coupling is zero carries no bond.
 *  - Bin geometry: S = sum over bonds of |J|. E lies in [-S, S] with E = S (mod 2); bin
 *    e = (E + S) / 2 in [0, S]. M lies in [-N, N] with M = N (mod 2); bin m = (M + N) / 2,
 *    the number of up spins. g is stored E-major: g[e * (N + 1) + m].
 *  - Thermodynamics: H = E - h*M (Eq. 1), Z = sum over states of exp(-H/T) (Eq. 2), k_B = 1.
 *    <E> denotes <H>, C = Var(H) / T^2, chi = Var(M) / T, all per system.
 *
 * Methods for g: oracle_g_edges (the definition, bond by bond), oracle_g_masks (the mask and
 * popcount form of Sec. 3a-3c), oracle_g_frontier (a transfer matrix over the site order) and
 * oracle_g_frontier_cut (the same, for every configuration of a cut set of spins). All four are
 * pinned by the tests against Table 1 (Sec. 4), closed forms and brute force.
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

#define ORC_OK 0
#define ORC_ERR_INVALID 1
#define ORC_ERR_TOO_LARGE 2
#define ORC_ERR_NOMEM 3

/* ------------------------------------------------------------------------------------------
 * Dense symmetric coupling matrix K[i*n + j] from an edge list, duplicates summed.
 * ---------------------------------------------------------------------------------------- */
static int build_couplings(int n, int64_t n_edges, const int32_t* ei, const int32_t* ej,
                           const int32_t* J, int64_t* K) {
    if (n < 1 || n > 64) return ORC_ERR_INVALID;
    memset(K, 0, sizeof(int64_t) * (size_t)n * (size_t)n);
    for (int64_t b = 0; b < n_edges; ++b) {
        int i = ei[b], j = ej[b];
        if (i < 0 || j < 0 || i >= n || j >= n || i == j) return ORC_ERR_INVALID;
        K[(size_t)i * n + j] += J[b];
        K[(size_t)j * n + i] += J[b];
    }
    return ORC_OK;
}

static int64_t total_abs_coupling(int n, const int64_t* K) {
    int64_t S = 0;
    for (int i = 0; i < n; ++i)
        for (int j = i + 1; j < n; ++j) S += llabs(K[(size_t)i * n + j]);
    return S;
}

/* Bin geometry of the table g for a graph (see the header comment). */
int oracle_bins(int n, int64_t n_edges, const int32_t* ei, const int32_t* ej, const int32_t* J,
                int64_t* e_min, int64_t* n_e, int64_t* n_m) {
    int64_t* K = (int64_t*)malloc(sizeof(int64_t) * 64 * 64);
    if (!K) return ORC_ERR_NOMEM;
    int rc = build_couplings(n, n_edges, ei, ej, J, K);
    if (rc == ORC_OK) {
        int64_t S = total_abs_coupling(n, K);
        *e_min = -S;
        *n_e = S + 1;
        *n_m = (int64_t)n + 1;
    }
    free(K);
    return rc;
}

/* ------------------------------------------------------------------------------------------
 * O0: the definition written out. For every configuration s in [s_lo, s_hi): read the spins
 * from the bits (Sec. 3a), sum -J S_i S_j over every bond once (Eq. 1), sum the spins for M
 * (Sec. 2), and add one to g at (E, M) (Sec. 2: the degeneracy of M over E).
 * g must hold (S + 1) * (n + 1) entries; it is accumulated into, not cleared.
 * ---------------------------------------------------------------------------------------- */
int oracle_g_edges(int n, int64_t n_edges, const int32_t* ei, const int32_t* ej, const int32_t* J,
                   uint64_t s_lo, uint64_t s_hi, int64_t* g) {
    int64_t K[64 * 64];
    int rc = build_couplings(n, n_edges, ei, ej, J, K);
    if (rc != ORC_OK) return rc;
    if (n > 62) return ORC_ERR_TOO_LARGE;
    uint64_t total = (uint64_t)1 << n;
    if (s_lo > s_hi || s_hi > total) return ORC_ERR_INVALID;
    const int64_t S = total_abs_coupling(n, K);
    /* bond list (i < j, K != 0) */
    int bi[64 * 63 / 2], bj[64 * 63 / 2];
    int64_t bJ[64 * 63 / 2];
    int nb = 0;
    for (int i = 0; i < n; ++i)
        for (int j = i + 1; j < n; ++j)
            if (K[i * n + j] != 0) { bi[nb] = i; bj[nb] = j; bJ[nb] = K[i * n + j]; ++nb; }
    for (uint64_t s = s_lo; s < s_hi; ++s) {
        int spin[64];
        int64_t M = 0;
        for (int i = 0; i < n; ++i) {
            spin[i] = ((s >> i) & 1u) ? +1 : -1;
            M += spin[i];
        }
        int64_t E = 0;
        for (int b = 0; b < nb; ++b) E -= bJ[b] * spin[bi[b]] * spin[bj[b]];
        int64_t e = (E + S) / 2, m = (M + n) / 2;
        g[e * (n + 1) + m] += 1;
    }
    return ORC_OK;
}

/* ------------------------------------------------------------------------------------------
 * O1: the same table from bit operations on the whole configuration word, in the manner of
 * Sec. 3a-3c: M from the number of units of the word (Sec. 3a); the exchange energy from
 * counting, for every spin k and every coupling value v on its forward bonds (partners j > k),
 * how many partners agree with spin k -- XOR of the word with spin k spread over all bits,
 * NOT, mask to the partners, count the units (Sec. 3b steps 1-3, Sec. 3c steps 2-5). A bond
 * with coupling v contributes -v when its two spins agree and +v otherwise, which for v = 1
 * on a periodic Z = 4 lattice is the paper's E_tot = 2(-En + N) (Sec. 3c).
 * Every configuration is evaluated from scratch (no Gray order, no incremental update).
 * threads > 1 splits [s_lo, s_hi) into contiguous pieces over OpenMP threads, each with its
 * own table, summed at the end.
 * ---------------------------------------------------------------------------------------- */
typedef struct {
    int k;           /* the spin owning these forward bonds */
    int64_t v;       /* coupling value on them */
    uint64_t mask;   /* partners j > k with K_kj == v */
    int deg;         /* number of partners in mask */
} fwd_group;

static int build_forward_groups(int n, const int64_t* K, fwd_group* out) {
    int ng = 0;
    for (int k = 0; k < n; ++k) {
        for (int j = k + 1; j < n; ++j) {
            int64_t v = K[k * n + j];
            if (v == 0) continue;
            int found = -1;
            for (int t = 0; t < ng; ++t)
                if (out[t].k == k && out[t].v == v) { found = t; break; }
            if (found < 0) {
                out[ng].k = k; out[ng].v = v; out[ng].mask = 0; out[ng].deg = 0;
                found = ng++;
            }
            out[found].mask |= (uint64_t)1 << j;
            out[found].deg += 1;
        }
    }
    return ng;
}

static int popcount64(uint64_t x) {
    /* Kernighan's loop, as quoted in Sec. 3a: clear the lowest set bit until none is left. */
    int c = 0;
    while (x) { x &= x - 1; ++c; }
    return c;
}

static void masks_range(int n, int64_t S, const fwd_group* grp, int ng, uint64_t lo, uint64_t hi,
                        int64_t* g) {
    for (uint64_t s = lo; s < hi; ++s) {
        int up = popcount64(s);
        int64_t E = 0;
        for (int t = 0; t < ng; ++t) {
            uint64_t spread = ((s >> grp[t].k) & 1u) ? ~(uint64_t)0 : 0;  /* spin k on every bit */
            uint64_t agree = ~(s ^ spread) & grp[t].mask;                  /* XOR, NOT, mask */
            int a = popcount64(agree);
            E += -grp[t].v * (int64_t)a + grp[t].v * (int64_t)(grp[t].deg - a);
        }
        g[((E + S) / 2) * (n + 1) + up] += 1;
    }
}

int oracle_g_masks(int n, int64_t n_edges, const int32_t* ei, const int32_t* ej, const int32_t* J,
                   uint64_t s_lo, uint64_t s_hi, int threads, int64_t* g) {
    int64_t K[64 * 64];
    int rc = build_couplings(n, n_edges, ei, ej, J, K);
    if (rc != ORC_OK) return rc;
    if (n > 62) return ORC_ERR_TOO_LARGE;
    uint64_t total = (uint64_t)1 << n;
    if (s_lo > s_hi || s_hi > total) return ORC_ERR_INVALID;
    const int64_t S = total_abs_coupling(n, K);
    fwd_group* grp = (fwd_group*)malloc(sizeof(fwd_group) * 64 * 63 / 2);
    if (!grp) return ORC_ERR_NOMEM;
    int ng = build_forward_groups(n, K, grp);
    const size_t nbins = (size_t)(S + 1) * (size_t)(n + 1);
    if (threads < 1) threads = 1;
    if (threads == 1) {
        masks_range(n, S, grp, ng, s_lo, s_hi, g);
        free(grp);
        return ORC_OK;
    }
    int64_t* part = (int64_t*)calloc((size_t)threads * nbins, sizeof(int64_t));
    if (!part) { free(grp); return ORC_ERR_NOMEM; }
    uint64_t span = s_hi - s_lo;
#pragma omp parallel for num_threads(threads) schedule(static, 1)
    for (int t = 0; t < threads; ++t) {
        uint64_t lo = s_lo + (span / threads) * t + (t < (int)(span % threads) ? t : span % threads);
        uint64_t len = span / threads + (t < (int)(span % threads) ? 1 : 0);
        masks_range(n, S, grp, ng, lo, lo + len, part + (size_t)t * nbins);
    }
    for (int t = 0; t < threads; ++t)
        for (size_t b = 0; b < nbins; ++b) g[b] += part[(size_t)t * nbins + b];
    free(part);
    free(grp);
    return ORC_OK;
}

/* ------------------------------------------------------------------------------------------
 * Frontier dynamic programme (a transfer matrix along the site order): an independent exact
 * method for g(E,M) that does not visit the 2^N configurations. Sites are added in index
 * order; a table indexed by the spins of the "active" sites (added sites that still have a
 * bond to a site not yet added) holds, for every partial energy of the bonds among added sites
 * and every number of up spins among them, the number of partial configurations. A site whose
 * last bond has been added is summed out. Cost grows as 2^(active sites); max_active bounds it.
 * Used to pin the other oracles and the enumerator on lattices too large for 2^N loops
 * (Sec. 2: g(E,M) is the degeneracy of the spin excess over the energy).
 *
 * frontier_rest runs the programme over the spins outside a cut set (cut bit i = spin i fixed
 * elsewhere), each carrying the cut's field f[v] as a one-spin energy term -f[v] S_v; with an
 * empty cut and f = 0 it is the plain programme of oracle_g_frontier.
 * ---------------------------------------------------------------------------------------- */
/* The rest's table out[e_r * (n_rest + 1) + m_r], e_r = (E_rest + S_rest) / 2, given the cut
 * field f[v] on every rest spin v; out holds (S_rest + 1) * (n_rest + 1) entries, overwritten. */
static int frontier_rest(int n, const int64_t* K, uint64_t cut, const int64_t* f, int64_t S_rest, int n_rest,
                         int max_active, int64_t* out) {
    int last_nb[64];                 /* largest rest neighbour index of each rest site, -1 if none */
    for (int i = 0; i < n; ++i) {
        last_nb[i] = -1;
        if ((cut >> i) & 1) continue;
        for (int j = 0; j < n; ++j)
            if (!((cut >> j) & 1) && K[i * n + j] != 0 && j > last_nb[i]) last_nb[i] = j;
    }
    int act[64];
    int na = 0, added = 0;
    int64_t Sp = 0;                  /* sum |J| over the bonds included so far (rest-rest and to the cut) */
    int64_t* tab = (int64_t*)calloc(1, sizeof(int64_t));
    if (!tab) return ORC_ERR_NOMEM;
    tab[0] = 1;                      /* empty configuration: energy 0 (e = 0 at Sp = 0), 0 up */
    /* layout: tab[(a * ne + e) * nm + m] with ne = Sp + 1 and nm = added + 1; bit t of a is the
     * spin of active site act[t] */
    for (int v = 0; v < n; ++v) {
        if ((cut >> v) & 1) continue;
        int64_t ne = Sp + 1, nm = added + 1;
        int64_t dS = 0;
        for (int t = 0; t < na; ++t) dS += llabs(K[act[t] * n + v]);
        for (int j = 0; j < n; ++j)
            if ((cut >> j) & 1) dS += llabs(K[v * n + j]);
        for (int u = 0; u < v; ++u)  /* every rest bond to an earlier rest site must reach an active one */
            if (!((cut >> u) & 1) && K[u * n + v] != 0) {
                int ok = 0;
                for (int t = 0; t < na; ++t) if (act[t] == u) ok = 1;
                if (!ok) { free(tab); return ORC_ERR_INVALID; }
            }
        int na1 = na + 1;
        if (na1 > max_active) { free(tab); return ORC_ERR_TOO_LARGE; }
        int64_t ne1 = Sp + dS + 1, nm1 = added + 2;
        int64_t* t1 = (int64_t*)calloc(((size_t)1 << na1) * (size_t)ne1 * (size_t)nm1, sizeof(int64_t));
        if (!t1) { free(tab); return ORC_ERR_NOMEM; }
        for (int64_t a = 0; a < ((int64_t)1 << na); ++a) {
            for (int sv = 0; sv < 2; ++sv) {
                int Sv = sv ? +1 : -1;
                int64_t dE = -f[v] * Sv;     /* the bonds to the cut, then to the active rest sites */
                for (int t = 0; t < na; ++t) {
                    int64_t Kuv = K[act[t] * n + v];
                    if (Kuv == 0) continue;
                    int Su = ((a >> t) & 1) ? +1 : -1;
                    dE -= Kuv * Su * Sv;
                }
                int64_t de = (dE + dS) / 2;   /* new e = (E + Sp + dS)/2 = e + (dE + dS)/2 */
                int64_t a1 = a | ((int64_t)sv << na);
                for (int64_t e = 0; e < ne; ++e)
                    for (int64_t m = 0; m < nm; ++m) {
                        int64_t c = tab[(a * ne + e) * nm + m];
                        if (c) t1[(a1 * ne1 + e + de) * nm1 + m + sv] += c;
                    }
            }
        }
        free(tab);
        tab = t1;
        act[na] = v;
        na = na1;
        Sp += dS;
        ++added;
        int keep[64], nk = 0;        /* sum out rest sites whose last rest bond is now in */
        for (int t = 0; t < na; ++t)
            if (last_nb[act[t]] > v) keep[nk++] = t;
        if (nk < na) {
            size_t sz2 = ((size_t)1 << nk) * (size_t)ne1 * (size_t)nm1;
            int64_t* t2 = (int64_t*)calloc(sz2, sizeof(int64_t));
            if (!t2) { free(tab); return ORC_ERR_NOMEM; }
            for (int64_t a = 0; a < ((int64_t)1 << na); ++a) {
                int64_t a2 = 0;
                for (int q = 0; q < nk; ++q) a2 |= ((a >> keep[q]) & 1) << q;
                for (int64_t x = 0; x < ne1 * nm1; ++x) t2[a2 * ne1 * nm1 + x] += tab[a * ne1 * nm1 + x];
            }
            free(tab);
            tab = t2;
            int act2[64];
            for (int q = 0; q < nk; ++q) act2[q] = act[keep[q]];
            for (int q = 0; q < nk; ++q) act[q] = act2[q];
            na = nk;
        }
    }
    if (Sp != S_rest || added != n_rest) { free(tab); return ORC_ERR_INVALID; }
    memcpy(out, tab, sizeof(int64_t) * (size_t)(S_rest + 1) * (size_t)(n_rest + 1));
    free(tab);
    return ORC_OK;
}

int oracle_g_frontier(int n, int64_t n_edges, const int32_t* ei, const int32_t* ej, const int32_t* J,
                      int max_active, int64_t* g) {
    int64_t K[64 * 64];
    int rc = build_couplings(n, n_edges, ei, ej, J, K);
    if (rc != ORC_OK) return rc;
    if (max_active > 24) max_active = 24;
    const int64_t S = total_abs_coupling(n, K);
    int64_t f[64];
    for (int v = 0; v < 64; ++v) f[v] = 0;
    int64_t* tab = (int64_t*)calloc((size_t)(S + 1) * (size_t)(n + 1), sizeof(int64_t));
    if (!tab) return ORC_ERR_NOMEM;
    rc = frontier_rest(n, K, 0, f, S, n, max_active, tab);
    if (rc == ORC_OK)
        for (int64_t x = 0; x < (S + 1) * (int64_t)(n + 1); ++x) g[x] += tab[x];
    free(tab);
    return rc;
}

/* ------------------------------------------------------------------------------------------
 * Frontier programme conditioned on a cut: an exact method for g(E,M) on lattices whose own
 * frontier is too wide (on a torus every cross-section is crossed twice). For every
 * configuration c of the spins in cut_mask (bit i = spin i), the other spins ("the rest") are
 * added in index order as in oracle_g_frontier: among themselves by their bonds, and to the cut
 * through the field f_v(c) = sum over cut spins j of J_vj S_j, a one-spin energy term -f_v S_v
 * (each bond to the cut counted once, as in Eq. 1). The rest's table over its energy and up
 * count is then shifted by the energy of the cut's own bonds and the cut's up count and added into
 * g: every configuration is exactly one c with one configuration of the rest, so the sum over c
 * counts every configuration once by its E and M (Sec. 2). Bins: e = (E + S)/2 splits as
 * (E_cut + S_cut)/2 + (E_rest + S_rest)/2, S_cut the sum of |J| over bonds inside the cut and
 * S_rest over the bonds touching the rest. threads > 1 hands the cut configurations to OpenMP
 * threads, each with its own table, summed at the end. The cut may be empty or hold every spin.
 * ---------------------------------------------------------------------------------------- */
int oracle_g_frontier_cut(int n, int64_t n_edges, const int32_t* ei, const int32_t* ej, const int32_t* J,
                          uint64_t cut_mask, int max_active, int threads, int64_t* g) {
    int64_t K[64 * 64];
    int rc = build_couplings(n, n_edges, ei, ej, J, K);
    if (rc != ORC_OK) return rc;
    if (n < 64 && (cut_mask >> n) != 0) return ORC_ERR_INVALID;
    if (max_active > 24) max_active = 24;
    int cut[64], k = 0;
    for (int i = 0; i < n; ++i) if ((cut_mask >> i) & 1) cut[k++] = i;
    if (k > 30) return ORC_ERR_TOO_LARGE;
    const int64_t S = total_abs_coupling(n, K);
    int64_t S_cut = 0;
    for (int a = 0; a < k; ++a)
        for (int b = a + 1; b < k; ++b) S_cut += llabs(K[cut[a] * n + cut[b]]);
    const int64_t S_rest = S - S_cut;
    const int n_rest = n - k;
    const size_t nbins = (size_t)(S + 1) * (size_t)(n + 1);
    const size_t rbins = (size_t)(S_rest + 1) * (size_t)(n_rest + 1);
    if (threads < 1) threads = 1;
    int64_t* part = (int64_t*)calloc((size_t)threads * nbins, sizeof(int64_t));
    int64_t* rest = (int64_t*)calloc((size_t)threads * rbins, sizeof(int64_t));
    if (!part || !rest) { free(part); free(rest); return ORC_ERR_NOMEM; }
    const int64_t n_cut_configs = (int64_t)1 << k;
    int status = ORC_OK;
#pragma omp parallel for num_threads(threads) schedule(dynamic, 1)
    for (int64_t c = 0; c < n_cut_configs; ++c) {
        int tid = 0;
#ifdef _OPENMP
        tid = omp_get_thread_num();
#endif
        int spin[64];
        for (int i = 0; i < n; ++i) spin[i] = 0;
        int up = 0;
        for (int a = 0; a < k; ++a) {
            spin[cut[a]] = ((c >> a) & 1) ? +1 : -1;
            up += (int)((c >> a) & 1);
        }
        int64_t E_cut = 0;           /* -J S_i S_j over the bonds inside the cut */
        for (int a = 0; a < k; ++a)
            for (int b = a + 1; b < k; ++b) E_cut -= K[cut[a] * n + cut[b]] * spin[cut[a]] * spin[cut[b]];
        int64_t f[64];               /* field of the cut on every rest spin */
        for (int v = 0; v < n; ++v) {
            f[v] = 0;
            if ((cut_mask >> v) & 1) continue;
            for (int a = 0; a < k; ++a) f[v] += K[v * n + cut[a]] * spin[cut[a]];
        }
        int64_t* rt = rest + (size_t)tid * rbins;
        int rc2 = frontier_rest(n, K, cut_mask, f, S_rest, n_rest, max_active, rt);
        if (rc2 != ORC_OK) {
#pragma omp critical
            status = rc2;
            continue;
        }
        const int64_t e_cut = (E_cut + S_cut) / 2;
        int64_t* gt = part + (size_t)tid * nbins;
        for (int64_t er = 0; er <= S_rest; ++er)
            for (int64_t mr = 0; mr <= n_rest; ++mr) {
                const int64_t cnt = rt[er * (n_rest + 1) + mr];
                if (cnt) gt[(e_cut + er) * (n + 1) + up + mr] += cnt;
            }
    }
    if (status == ORC_OK)
        for (int t = 0; t < threads; ++t)
            for (size_t b = 0; b < nbins; ++b) g[b] += part[(size_t)t * nbins + b];
    free(part);
    free(rest);
    return status;
}

/* ------------------------------------------------------------------------------------------
 * Thermodynamics from g by the definition: for every (T, h) point, Z = sum over bins of
 * g(E,M) exp(-(E - h M)/T) (Eq. 2 grouped by the degeneracy of Sec. 2). Every term is taken
 * relative to the largest log-weight ln g - H/T so nothing overflows; sums run in long double.
 * Means and variances are taken from the same weights, the variances about the mean (two
 * passes). Outputs per point p = iT * nh + ih: logZ, <H>, <M>, C = Var(H)/T^2, chi = Var(M)/T.
 * ---------------------------------------------------------------------------------------- */
int oracle_thermo(int n, int64_t e_min, int64_t n_e, const int64_t* g, int nT, const double* T,
                  int nh, const double* h, double* logZ, double* Emean, double* Mmean, double* C,
                  double* chi) {
    const int64_t n_m = (int64_t)n + 1;
    for (int it = 0; it < nT; ++it) {
        if (!(T[it] > 0)) return ORC_ERR_INVALID;
        for (int ih = 0; ih < nh; ++ih) {
            const long double t = T[it], f = h[ih];
            long double Lmax = -INFINITY;
            for (int64_t e = 0; e < n_e; ++e)
                for (int64_t m = 0; m < n_m; ++m) {
                    int64_t c = g[e * n_m + m];
                    if (c <= 0) continue;
                    long double E = (long double)(e_min + 2 * e), M = (long double)(-n + 2 * m);
                    long double lw = logl((long double)c) - (E - f * M) / t;
                    if (lw > Lmax) Lmax = lw;
                }
            long double Z = 0, sH = 0, sM = 0;
            for (int64_t e = 0; e < n_e; ++e)
                for (int64_t m = 0; m < n_m; ++m) {
                    int64_t c = g[e * n_m + m];
                    if (c <= 0) continue;
                    long double E = (long double)(e_min + 2 * e), M = (long double)(-n + 2 * m);
                    long double H = E - f * M;
                    long double w = expl(logl((long double)c) - H / t - Lmax);
                    Z += w; sH += w * H; sM += w * M;
                }
            long double mH = sH / Z, mM = sM / Z, vH = 0, vM = 0;
            for (int64_t e = 0; e < n_e; ++e)
                for (int64_t m = 0; m < n_m; ++m) {
                    int64_t c = g[e * n_m + m];
                    if (c <= 0) continue;
                    long double E = (long double)(e_min + 2 * e), M = (long double)(-n + 2 * m);
                    long double H = E - f * M;
                    long double w = expl(logl((long double)c) - H / t - Lmax);
                    vH += w * (H - mH) * (H - mH);
                    vM += w * (M - mM) * (M - mM);
                }
            vH /= Z; vM /= Z;
            const int64_t p = (int64_t)it * nh + ih;
            logZ[p] = (double)(Lmax + logl(Z));
            Emean[p] = (double)mH;
            Mmean[p] = (double)mM;
            C[p] = (double)(vH / (t * t));
            chi[p] = (double)(vM / t);
        }
    }
    return ORC_OK;
}

/* ------------------------------------------------------------------------------------------
 * Magnetisation statistics from g by the definition, for comparing finite systems with
 * measured magnetisation and for locating their ordering temperature (Sec. 1, Sec. 5). At h = 0
 * the mean magnetisation of a finite system is exactly zero (g is symmetric in M), so the
 * curves are given by the moments of |M| and M: per point p = iT * nh + ih, with weights
 * g(E,M) exp(-(E - h M)/T) taken relative to the largest log-weight and summed in long double,
 *   absM = <|M|>,  M2 = <M^2>,  M4 = <M^4>,  binder = 1 - <M^4> / (3 <M^2>^2),
 * the last being Binder's fourth-order cumulant (2/3 in a fully ordered state, 0 for Gaussian
 * fluctuations of M). binder is 0 when <M^2> = 0 (a system with no spins).
 * ---------------------------------------------------------------------------------------- */
int oracle_magnetisation(int n, int64_t e_min, int64_t n_e, const int64_t* g, int nT, const double* T,
                         int nh, const double* h, double* absM, double* M2, double* M4, double* binder) {
    const int64_t n_m = (int64_t)n + 1;
    for (int it = 0; it < nT; ++it) {
        if (!(T[it] > 0)) return ORC_ERR_INVALID;
        for (int ih = 0; ih < nh; ++ih) {
            const long double t = T[it], f = h[ih];
            long double Lmax = -INFINITY;
            for (int64_t e = 0; e < n_e; ++e)
                for (int64_t m = 0; m < n_m; ++m) {
                    int64_t c = g[e * n_m + m];
                    if (c <= 0) continue;
                    long double E = (long double)(e_min + 2 * e), M = (long double)(-n + 2 * m);
                    long double lw = logl((long double)c) - (E - f * M) / t;
                    if (lw > Lmax) Lmax = lw;
                }
            long double Z = 0, sA = 0, s2 = 0, s4 = 0;
            for (int64_t e = 0; e < n_e; ++e)
                for (int64_t m = 0; m < n_m; ++m) {
                    int64_t c = g[e * n_m + m];
                    if (c <= 0) continue;
                    long double E = (long double)(e_min + 2 * e), M = (long double)(-n + 2 * m);
                    long double w = expl(logl((long double)c) - (E - f * M) / t - Lmax);
                    Z += w;
                    sA += w * fabsl(M);
                    s2 += w * M * M;
                    s4 += w * M * M * M * M;
                }
            const int64_t p = (int64_t)it * nh + ih;
            const long double m2 = s2 / Z, m4 = s4 / Z;
            absM[p] = (double)(sA / Z);
            M2[p] = (double)m2;
            M4[p] = (double)m4;
            binder[p] = m2 > 0 ? (double)(1.0L - m4 / (3.0L * m2 * m2)) : 0.0;
        }
    }
    return ORC_OK;
}
