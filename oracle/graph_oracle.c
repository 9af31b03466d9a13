/*
 * graph_oracle.c -- plain, slow, single-threaded CPU reference of one
 * Swendsen-Wang sweep on an arbitrary lattice given as a list of
 * nearest-neighbour bonds (optionally diluted).
 *
 * TEST INFRASTRUCTURE ONLY, like pyro_oracle.c, with which it is compiled
 * into the oracle library (it uses that file's Philox streams, unit-vector
 * sampler, thresholds and sequential union-find).  It shares no source with
 * the CUDA library.
 *
 * What it follows (Soldatov, Nefedev, Komura, Okabe, arXiv:1612.08312):
 *   - Sec. 2: the SW program is lattice-generic once the table of each
 *     site's nearest neighbours is given; the Hamiltonian of Eq. 1 summed
 *     over the table's pairs;
 *   - Sec. 3.4 (Eq. 5-6): the simple-cubic lattice, coordination number
 *     six like the pyrochlore lattice, as the comparison lattice;
 *   - Sec. 4: diluted lattices (vacant sites, missing bonds) as the
 *     extension the paper names.
 *
 * Conventions that the paper leaves open (the same as the CUDA path's):
 *   - bond e of the list joins sites bond_i[e] and bond_j[e] (no self
 *     loops); its random-number id is e, so its 32-bit uniform is
 *     orc_bond_word(seed, sweep, e), and the pyrochlore lattice's own bond
 *     list ordered by its random-number ids gives the pyrochlore chain;
 *   - a neighbour table nbr[N][z] (-1 = no neighbour) gives the bond list
 *     of every slot (i, k) with i < nbr[i][k], in the order of (i, k);
 *   - the simple-cubic lattice of L^3 sites: site i = x + L (y + L z),
 *     bond 3 i + d joins i to its neighbour one step along +axis d
 *     (periodic), found here from the sites' positions;
 *   - dilution: a vacant site (site mask 0) holds a spin that takes no
 *     part in the dynamics: every bond that touches it is absent, it is a
 *     cluster of its own and it never flips; a bond with edge mask 0 is
 *     absent.  Absent bonds are never active and do not enter E;
 *   - E = -J sum over present bonds of s_i . s_j; m = |M| / N_occ with M
 *     summed over occupied sites (m = 0 when no site is occupied);
 *   - random start and flip bits as in pyro_oracle.c, by site index.
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

#define GORC_ISING 1
#define TAG_FLIP 2u
#define TAG_AXIS 3u
#define TAG_INIT 4u
#define INIT_SWEEP_FIELD 0xFFFFFFFFu

/* from pyro_oracle.c */
uint32_t orc_bond_word(uint64_t seed, uint32_t sweep_field, uint64_t b);
uint64_t orc_prob_threshold(double p);
uint64_t orc_threshold(double beta, double J);
uint32_t orc_stream_bit(uint64_t seed, uint32_t sweep_field, uint32_t tag, uint64_t x);
int orc_unit_vector(uint64_t seed, uint32_t sweep_field, uint32_t tag, uint64_t call_base, int n, double r[3]);
int orc_clusters(int64_t nsites, int64_t nbonds, const int32_t *bi, const int32_t *bj, const uint8_t *active,
                 int32_t *labels);

/* ------------------------------------------------------------------------
 * Bond lists.
 * ---------------------------------------------------------------------- */

/* Bond list of a neighbour table (Sec. 2): slot (i, k) with
 * i < nbr[i z + k] is a bond, in the order of (i, k).  The table must be
 * symmetric: j appears in i's row as often as i appears in j's row.
 * Returns the number of bonds (bi, bj may be NULL to count only), or -1 if
 * an entry is out of range, names its own site, or the table is not
 * symmetric. */
int64_t gorc_edges_from_table(int64_t N, int z, const int32_t *nbr, int32_t *bi, int32_t *bj)
{
    int64_t E = 0;
    for (int64_t i = 0; i < N; ++i)
        for (int k = 0; k < z; ++k) {
            int32_t j = nbr[i * z + k];
            if (j < 0) continue;
            if (j >= N || j == i) return -1;
            /* multiplicity of i in j's row must equal that of j in i's row */
            int a = 0, b = 0;
            for (int q = 0; q < z; ++q) {
                if (nbr[i * z + q] == j) ++a;
                if (nbr[(int64_t)j * z + q] == i) ++b;
            }
            if (a != b) return -1;
            if (i < j) {
                if (bi) { bi[E] = (int32_t)i; bj[E] = j; }
                ++E;
            }
        }
    return E;
}

/* Simple-cubic L^3 lattice (Sec. 3.4), periodic: 3 L^3 bonds.  Each site's
 * position is (x, y, z) with i = x + L (y + L z); bond 3 i + d goes to the
 * site whose position is one step further along axis d, found by searching
 * the positions (not by index arithmetic). */
int gorc_sc_edges(int L, int32_t *bi, int32_t *bj)
{
    if (L < 2) return -1;
    const int64_t N = (int64_t)L * L * L;
    int32_t *pos = (int32_t *)malloc((size_t)N * 3 * sizeof(int32_t));
    int32_t *at = (int32_t *)malloc((size_t)N * sizeof(int32_t));  /* position key -> site */
    if (!pos || !at) { free(pos); free(at); return -1; }
    for (int64_t i = 0; i < N; ++i) {
        pos[3 * i + 0] = (int32_t)(i % L);
        pos[3 * i + 1] = (int32_t)((i / L) % L);
        pos[3 * i + 2] = (int32_t)(i / ((int64_t)L * L));
    }
    for (int64_t i = 0; i < N; ++i) at[i] = -1;
    for (int64_t i = 0; i < N; ++i) {
        /* position key in z-major order, independent of the index formula */
        int64_t key = ((int64_t)pos[3 * i + 2] * L + pos[3 * i + 1]) * L + pos[3 * i + 0];
        at[key] = (int32_t)i;
    }
    for (int64_t i = 0; i < N; ++i)
        for (int d = 0; d < 3; ++d) {
            int32_t q[3] = {pos[3 * i + 0], pos[3 * i + 1], pos[3 * i + 2]};
            q[d] = (q[d] + 1) % L;
            int64_t key = ((int64_t)q[2] * L + q[1]) * L + q[0];
            bi[3 * i + d] = (int32_t)i;
            bj[3 * i + d] = at[key];
        }
    free(pos);
    free(at);
    return 0;
}

/* ------------------------------------------------------------------------
 * State.
 * ---------------------------------------------------------------------- */
typedef struct { double s, c; } gsum;

static void gsum_add(gsum *a, double x)
{
    double t = a->s + x;
    if (fabs(a->s) >= fabs(x)) a->c += (a->s - t) + x;
    else a->c += (x - t) + a->s;
    a->s = t;
}

typedef struct gorc {
    int model, ncomp;
    int64_t N, NB, Nocc;
    uint64_t seed;
    double J;
    uint64_t sweep;
    int32_t *bi, *bj;
    uint8_t *occ;       /* site occupied */
    uint8_t *present;   /* bond present: edge mask and both ends occupied */
    int8_t *sigma;      /* Ising spins */
    double *spin;       /* n-vector spins, SoA: spin[k N + i] */
    double *proj;
    int32_t *label;
    uint8_t *active;
    double axis[3];
    gsum acc[5];
    uint64_t count;
} gorc;

void gorc_free(gorc *h)
{
    if (!h) return;
    free(h->bi); free(h->bj); free(h->occ); free(h->present); free(h->sigma); free(h->spin);
    free(h->proj); free(h->label); free(h->active);
    free(h);
}

/* A lattice of N sites and NB bonds; site_mask / edge_mask may be NULL
 * (all present).  start: 0 ordered, 1 random (as pyro_oracle.c). */
gorc *gorc_new(int64_t N, int64_t NB, const int32_t *bi, const int32_t *bj, const uint8_t *site_mask,
               const uint8_t *edge_mask, int model, uint64_t seed, int start, double J)
{
    if (N < 1 || NB < 0 || model < 1 || model > 3) return NULL;
    for (int64_t e = 0; e < NB; ++e)
        if (bi[e] < 0 || bi[e] >= N || bj[e] < 0 || bj[e] >= N || bi[e] == bj[e]) return NULL;
    gorc *h = (gorc *)calloc(1, sizeof(gorc));
    if (!h) return NULL;
    h->model = model; h->ncomp = model; h->N = N; h->NB = NB; h->seed = seed; h->J = J;
    h->bi = (int32_t *)malloc((size_t)(NB ? NB : 1) * sizeof(int32_t));
    h->bj = (int32_t *)malloc((size_t)(NB ? NB : 1) * sizeof(int32_t));
    h->occ = (uint8_t *)malloc((size_t)N);
    h->present = (uint8_t *)malloc((size_t)(NB ? NB : 1));
    h->active = (uint8_t *)calloc((size_t)(NB ? NB : 1), 1);
    h->label = (int32_t *)malloc((size_t)N * sizeof(int32_t));
    if (model == GORC_ISING) h->sigma = (int8_t *)malloc((size_t)N);
    else {
        h->spin = (double *)malloc((size_t)N * model * sizeof(double));
        h->proj = (double *)malloc((size_t)N * sizeof(double));
    }
    if (!h->bi || !h->bj || !h->occ || !h->present || !h->active || !h->label ||
        (model == GORC_ISING ? !h->sigma : (!h->spin || !h->proj))) { gorc_free(h); return NULL; }
    memcpy(h->bi, bi, (size_t)NB * sizeof(int32_t));
    memcpy(h->bj, bj, (size_t)NB * sizeof(int32_t));
    h->Nocc = 0;
    for (int64_t i = 0; i < N; ++i) {
        h->occ[i] = site_mask ? (site_mask[i] != 0) : 1;
        h->Nocc += h->occ[i];
        h->label[i] = (int32_t)i;
    }
    for (int64_t e = 0; e < NB; ++e)
        h->present[e] = (uint8_t)((edge_mask ? edge_mask[e] != 0 : 1) && h->occ[bi[e]] && h->occ[bj[e]]);
    for (int64_t i = 0; i < N; ++i) {
        if (model == GORC_ISING) {
            h->sigma[i] = (start && orc_stream_bit(seed, INIT_SWEEP_FIELD, TAG_INIT, (uint64_t)i)) ? -1 : 1;
        } else {
            double r[3] = {1.0, 0.0, 0.0};
            if (start) orc_unit_vector(seed, INIT_SWEEP_FIELD, TAG_INIT, (uint64_t)i << 8, model, r);
            for (int k = 0; k < model; ++k) h->spin[k * N + i] = r[k];
        }
    }
    return h;
}

/* Eq. 1 energy over the present bonds and Eq. 2 moments of m = |M|/N_occ. */
void gorc_measure(const gorc *h, double *E, double *m2, double *m4, double *Mvec)
{
    const int64_t N = h->N;
    double m;
    if (h->model == GORC_ISING) {
        int64_t M = 0, sat = 0, anti = 0;
        for (int64_t i = 0; i < N; ++i)
            if (h->occ[i]) M += h->sigma[i];
        for (int64_t e = 0; e < h->NB; ++e) {
            if (!h->present[e]) continue;
            if (h->sigma[h->bi[e]] == h->sigma[h->bj[e]]) ++sat; else ++anti;
        }
        *E = -h->J * (double)(sat - anti);
        m = h->Nocc ? fabs((double)M) / (double)h->Nocc : 0.0;
        if (Mvec) { Mvec[0] = (double)M; Mvec[1] = 0.0; Mvec[2] = 0.0; }
    } else {
        const int n = h->ncomp;
        double Mk[3] = {0.0, 0.0, 0.0};
        for (int k = 0; k < n; ++k)
            for (int64_t i = 0; i < N; ++i)
                if (h->occ[i]) Mk[k] += h->spin[k * N + i];
        double e = 0.0;
        for (int64_t b = 0; b < h->NB; ++b) {
            if (!h->present[b]) continue;
            int64_t i = h->bi[b], j = h->bj[b];
            double d = h->spin[i] * h->spin[j];
            for (int k = 1; k < n; ++k) d += h->spin[k * N + i] * h->spin[k * N + j];
            e += d;
        }
        *E = -h->J * e;
        double msq = Mk[0] * Mk[0];
        for (int k = 1; k < n; ++k) msq += Mk[k] * Mk[k];
        m = h->Nocc ? sqrt(msq) / (double)h->Nocc : 0.0;
        if (Mvec) { Mvec[0] = Mk[0]; Mvec[1] = Mk[1]; Mvec[2] = Mk[2]; }
    }
    *m2 = m * m;
    *m4 = (*m2) * (*m2);
}

/* One Swendsen-Wang sweep on the bond list (Sec. 2; Wolff embedding for
 * n > 1), in the order: bond activation, clusters, cluster flips,
 * measurement. */
static void gsweep_once(gorc *h, double beta, double *trace)
{
    const int64_t N = h->N, NB = h->NB;
    const uint32_t sw = (uint32_t)h->sweep;
    const int n = h->ncomp;

    /* 1. bond activation: present bonds only, bond id = list position */
    if (h->model == GORC_ISING) {
        const uint64_t thr = orc_threshold(beta, h->J);
        for (int64_t e = 0; e < NB; ++e) {
            int act = 0;
            if (h->present[e] && h->sigma[h->bi[e]] == h->sigma[h->bj[e]])
                act = ((uint64_t)orc_bond_word(h->seed, sw, (uint64_t)e) < thr);
            h->active[e] = (uint8_t)act;
        }
    } else {
        orc_unit_vector(h->seed, sw, TAG_AXIS, 0, n, h->axis);
        for (int64_t i = 0; i < N; ++i) {
            double p = h->spin[i] * h->axis[0];
            for (int k = 1; k < n; ++k) p = p + h->spin[k * N + i] * h->axis[k];
            h->proj[i] = p;
        }
        const double K2 = 2.0 * beta * h->J;
        for (int64_t e = 0; e < NB; ++e) {
            int act = 0;
            if (h->present[e]) {
                double x = h->proj[h->bi[e]] * h->proj[h->bj[e]];
                if (x > 0.0) {
                    double prob = -expm1(-(K2 * x));
                    act = ((uint64_t)orc_bond_word(h->seed, sw, (uint64_t)e) < orc_prob_threshold(prob));
                }
            }
            h->active[e] = (uint8_t)act;
        }
    }

    /* 2. clusters of the active bonds: canonical label = minimum site */
    orc_clusters(N, NB, h->bi, h->bj, h->active, h->label);

    /* 3-4. occupied sites flip with their cluster's bit */
    for (int64_t i = 0; i < N; ++i) {
        if (!h->occ[i]) continue;
        if (!orc_stream_bit(h->seed, sw, TAG_FLIP, (uint64_t)h->label[i])) continue;
        if (h->model == GORC_ISING) {
            h->sigma[i] = (int8_t)(-h->sigma[i]);
        } else {
            double d2 = 2.0 * h->proj[i];
            double s[3];
            for (int k = 0; k < n; ++k) s[k] = h->spin[k * N + i] - d2 * h->axis[k];
            double q = s[0] * s[0];
            for (int k = 1; k < n; ++k) q = q + s[k] * s[k];
            q = sqrt(q);
            for (int k = 0; k < n; ++k) h->spin[k * N + i] = s[k] / q;
        }
    }

    /* 5. measurement and compensated accumulation */
    double E, m2, m4, Mv[3];
    gorc_measure(h, &E, &m2, &m4, Mv);
    gsum_add(&h->acc[0], E);
    gsum_add(&h->acc[1], E * E);
    gsum_add(&h->acc[2], m2);
    gsum_add(&h->acc[3], m4);
    gsum_add(&h->acc[4], sqrt(m2));
    h->count += 1;
    if (trace) { trace[0] = E; trace[1] = m2; trace[2] = m4; trace[3] = Mv[0]; }
    h->sweep += 1;
}

int gorc_sweep(gorc *h, double beta, int64_t n, double *trace)
{
    if (!h || n < 0 || !(beta >= 0.0)) return -1;
    for (int64_t s = 0; s < n; ++s) gsweep_once(h, beta, trace ? trace + 4 * s : NULL);
    return 0;
}

void gorc_stats(const gorc *h, double out[6])
{
    out[0] = (double)h->count;
    for (int k = 0; k < 5; ++k) out[k + 1] = h->acc[k].s + h->acc[k].c;
}

void gorc_reset_stats(gorc *h)
{
    memset(h->acc, 0, sizeof(h->acc));
    h->count = 0;
}

int64_t gorc_num_sites(const gorc *h) { return h->N; }
int64_t gorc_num_bonds(const gorc *h) { return h->NB; }
uint64_t gorc_get_sweep(const gorc *h) { return h->sweep; }
void gorc_set_sweep(gorc *h, uint64_t s) { h->sweep = s; }
void gorc_get_labels(const gorc *h, int32_t *out) { memcpy(out, h->label, (size_t)h->N * sizeof(int32_t)); }
void gorc_get_active(const gorc *h, uint8_t *out) { memcpy(out, h->active, (size_t)h->NB); }
void gorc_get_axis(const gorc *h, double out[3]) { memcpy(out, h->axis, sizeof(h->axis)); }

/* Spins in site order: Ising int8 +-1; n > 1 doubles, site-major (N x n). */
void gorc_get_spins(const gorc *h, void *out)
{
    if (h->model == GORC_ISING) { memcpy(out, h->sigma, (size_t)h->N); return; }
    double *o = (double *)out;
    for (int64_t i = 0; i < h->N; ++i)
        for (int k = 0; k < h->ncomp; ++k) o[i * h->ncomp + k] = h->spin[k * h->N + i];
}

void gorc_set_spins(gorc *h, const void *in)
{
    if (h->model == GORC_ISING) { memcpy(h->sigma, in, (size_t)h->N); return; }
    const double *s = (const double *)in;
    for (int64_t i = 0; i < h->N; ++i)
        for (int k = 0; k < h->ncomp; ++k) h->spin[k * h->N + i] = s[i * h->ncomp + k];
}
