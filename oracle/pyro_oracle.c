/*
 * pyro_oracle.c -- plain, slow, single-threaded CPU reference of one
 * Swendsen-Wang sweep on the ferromagnetic pyrochlore lattice.
 *
 * TEST INFRASTRUCTURE ONLY.  This file is the oracle that the CUDA library
 * is checked against.  Only the test suite, the smoke check and the CPU
 * baseline leg of the benchmark load it.  It shares no source with the CUDA
 * path and includes none of its headers.
 *
 * What it follows (Soldatov, Nefedev, Komura, Okabe, arXiv:1612.08312):
 *   - Sec. 2: the 16-site cubic unit cell, L x L x L cells, periodic
 *     boundaries, N = 16 L^3, coordination number six.
 *   - Eq. 1: H = -J sum_<ij> s_i . s_j with unit n-vectors, n = 1, 2, 3.
 *   - Sec. 1-2: the Swendsen-Wang multi-cluster update, with Wolff's
 *     embedded-cluster (reflection) form for n = 2, 3.
 *   - Eq. 2: the moment ratio U = <m^4>/<m^2>^2 with m = M/N.
 *
 * Conventions that the paper leaves open:
 *   - site index i = 16*(x + L*(y + L*z)) + 4*f + mu, position (quarter
 *     units) 4*(x,y,z) + A_f + B_mu;
 *   - bonds grouped by tetrahedron: bond 12*r + k, r = i >> 2 the FCC point,
 *     k = 0..5 the vertex pairs (0,1) (0,2) (0,3) (1,2) (1,3) (2,3) of the
 *     "up" tetrahedron of r, k = 6..11 the same pairs of the "down"
 *     tetrahedron whose basis-0 vertex is site 4r;
 *   - the random-number id of a bond of cell c, FCC sub-point f:
 *     b = 48 c + 16 g + 4 f + q with (g, q) = (0,0) up (0,1), (0,1) up (1,2),
 *     (0,2) up (2,3), (0,3) up (0,3), (1,0) up (0,2), (1,1) up (1,3),
 *     (1,2) down (0,2), (1,3) down (1,3), (2,0) down (0,1), (2,1) down
 *     (1,2), (2,2) down (2,3), (2,3) down (0,3);
 *   - random numbers from Philox4x32-10 keyed by the seed, counter
 *     (j_lo, j_hi, sweep, tag).  A call yields 128 bits, read as sixteen
 *     bytes (byte t = bits 8 (t & 3) .. of output word t >> 2), four words,
 *     or 128 single bits (bit t = bit t & 31 of output word t >> 5);
 *   - bond b's 32-bit uniform w_b: top 8 bits = byte (b & 15) of BOND call
 *     b >> 4, low 24 bits = low 24 bits of word (b & 3) of TIE call b >> 2;
 *   - one flip bit per cluster: bit (root & 127) of FLIP call root >> 7;
 *   - canonical cluster label = minimum site index of the cluster.
 *
 * The nearest-neighbour table is found GEOMETRICALLY (every lattice point at
 * squared distance 2 in quarter units), not from a closed form.  Union-find
 * is sequential.  Floating point is IEEE double, compiled with
 * -ffp-contract=off so that no multiply-add is fused.
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

#define ORC_ISING 1
#define ORC_XY 2
#define ORC_HEIS 3

#define TAG_BOND 1u
#define TAG_FLIP 2u
#define TAG_AXIS 3u
#define TAG_INIT 4u
#define TAG_TIE 5u
#define INIT_SWEEP_FIELD 0xFFFFFFFFu
#define MAX_AXIS_ATTEMPTS 256

/* ------------------------------------------------------------------------
 * Philox4x32-10, written from Salmon, Moraes, Dror and Shaw, "Parallel
 * random numbers: as easy as 1, 2, 3" (SC'11): ten rounds of the Philox
 * S-box on a 4-word counter with a 2-word key bumped by the Weyl constants
 * between rounds.
 * ---------------------------------------------------------------------- */
void orc_philox(const uint32_t ctr_in[4], const uint32_t key_in[2], uint32_t out[4])
{
    uint32_t c0 = ctr_in[0], c1 = ctr_in[1], c2 = ctr_in[2], c3 = ctr_in[3];
    uint32_t k0 = key_in[0], k1 = key_in[1];
    for (int round = 0; round < 10; ++round) {
        if (round > 0) {
            k0 += 0x9E3779B9u;
            k1 += 0xBB67AE85u;
        }
        uint64_t prodA = (uint64_t)0xD2511F53u * (uint64_t)c0;
        uint64_t prodB = (uint64_t)0xCD9E8D57u * (uint64_t)c2;
        uint32_t hiA = (uint32_t)(prodA >> 32), loA = (uint32_t)prodA;
        uint32_t hiB = (uint32_t)(prodB >> 32), loB = (uint32_t)prodB;
        uint32_t n0 = hiB ^ c1 ^ k0;
        uint32_t n1 = loB;
        uint32_t n2 = hiA ^ c3 ^ k1;
        uint32_t n3 = loA;
        c0 = n0; c1 = n1; c2 = n2; c3 = n3;
    }
    out[0] = c0; out[1] = c1; out[2] = c2; out[3] = c3;
}

static void stream_call(uint64_t seed, uint32_t sweep_field, uint32_t tag, uint64_t j, uint32_t out[4])
{
    uint32_t ctr[4] = {(uint32_t)j, (uint32_t)(j >> 32), sweep_field, tag};
    uint32_t key[2] = {(uint32_t)seed, (uint32_t)(seed >> 32)};
    orc_philox(ctr, key, out);
}

/* Byte x of the stream (seed, sweep field, tag): byte x & 15 of the Philox
 * call with call index x >> 4. */
static uint32_t stream_byte(uint64_t seed, uint32_t sweep_field, uint32_t tag, uint64_t x)
{
    uint32_t out[4];
    stream_call(seed, sweep_field, tag, x >> 4, out);
    return (out[(x & 15) >> 2] >> (8 * (x & 3))) & 0xFFu;
}

/* Word x of the stream: output word x & 3 of the call with index x >> 2. */
static uint32_t stream_word(uint64_t seed, uint32_t sweep_field, uint32_t tag, uint64_t x)
{
    uint32_t out[4];
    stream_call(seed, sweep_field, tag, x >> 2, out);
    return out[x & 3];
}

/* Bit x of the stream: bit x & 127 of the Philox call with index x >> 7. */
static uint32_t stream_bit(uint64_t seed, uint32_t sweep_field, uint32_t tag, uint64_t x)
{
    uint32_t out[4];
    stream_call(seed, sweep_field, tag, x >> 7, out);
    return (out[(x & 127) >> 5] >> (x & 31)) & 1u;
}

/* The 32-bit uniform of the bond with random-number id b in a sweep. */
uint32_t orc_bond_word(uint64_t seed, uint32_t sweep_field, uint64_t b)
{
    return (stream_byte(seed, sweep_field, TAG_BOND, b) << 24) |
           (stream_word(seed, sweep_field, TAG_TIE, b) & 0xFFFFFFu);
}

/* Random-number id of bond 12 r + k (see the header comment). */
static const int RNG_G[12] = {0, 1, 0, 0, 1, 0, 2, 1, 2, 2, 1, 2};
static const int RNG_Q[12] = {0, 0, 3, 1, 1, 2, 0, 2, 3, 1, 3, 2};

uint64_t orc_bond_rng_id(uint64_t bond)
{
    uint64_t r = bond / 12, k = bond % 12;
    uint64_t c = r >> 2, f = r & 3;
    return 48 * c + 16 * (uint64_t)RNG_G[k] + 4 * f + (uint64_t)RNG_Q[k];
}

/* Threshold of a bond with activation probability p: the bond is active iff
 * its uniform w < floor(p * 2^32).  Returned in 64 bits so that p = 1 gives
 * 2^32 (every word below it). */
static uint64_t prob_threshold(double p)
{
    if (!(p > 0.0)) return 0;
    double t = floor(p * 4294967296.0);
    if (t >= 4294967296.0) return (uint64_t)1 << 32;
    return (uint64_t)t;
}

/* Exported forms of the two helpers above, for graph_oracle.c. */
uint64_t orc_prob_threshold(double p) { return prob_threshold(p); }
uint32_t orc_stream_bit(uint64_t seed, uint32_t sweep_field, uint32_t tag, uint64_t x)
{
    return stream_bit(seed, sweep_field, tag, x);
}

/* Ising: a satisfied bond is active with p = 1 - exp(-2 beta J)
 * (Swendsen-Wang bond probability; SW87 as cited in Sec. 1). */
uint64_t orc_threshold(double beta, double J)
{
    return prob_threshold(-expm1(-2.0 * beta * J));
}

/* Uniform random unit vector for the embedded-cluster axis (n = 2, 3) and
 * for random continuous-spin starts.  Rejection sampling in the square:
 * u0, u1 = signed words scaled by 2^-31, s = u0^2 + u1^2, accept 0 < s < 1.
 * n = 2: r = (u0, u1)/sqrt(s).  n = 3: Marsaglia (1972),
 * r = (2 u0 sqrt(1-s), 2 u1 sqrt(1-s), 1 - 2 s).
 * Attempt a uses Philox call index call_base + a (word pair 0, 1).
 * Returns the number of attempts used; if none of MAX_AXIS_ATTEMPTS is
 * accepted (probability about 1e-170) r = e_0. */
int orc_unit_vector(uint64_t seed, uint32_t sweep_field, uint32_t tag, uint64_t call_base,
                    int n, double r[3])
{
    uint32_t key[2] = {(uint32_t)seed, (uint32_t)(seed >> 32)};
    for (int a = 0; a < MAX_AXIS_ATTEMPTS; ++a) {
        uint64_t j = call_base + (uint64_t)a;
        uint32_t ctr[4] = {(uint32_t)j, (uint32_t)(j >> 32), sweep_field, tag};
        uint32_t w[4];
        orc_philox(ctr, key, w);
        double u0 = (double)(int32_t)w[0] * (1.0 / 2147483648.0);
        double u1 = (double)(int32_t)w[1] * (1.0 / 2147483648.0);
        double s = u0 * u0 + u1 * u1;
        if (s > 0.0 && s < 1.0) {
            if (n == 2) {
                double q = sqrt(s);
                r[0] = u0 / q;
                r[1] = u1 / q;
                r[2] = 0.0;
            } else {
                double t = sqrt(1.0 - s);
                r[0] = 2.0 * u0 * t;
                r[1] = 2.0 * u1 * t;
                r[2] = 1.0 - 2.0 * s;
            }
            return a + 1;
        }
    }
    r[0] = 1.0; r[1] = 0.0; r[2] = 0.0;
    return MAX_AXIS_ATTEMPTS;
}

/* ------------------------------------------------------------------------
 * Lattice, built by geometry (Sec. 2: 16-site cubic cell, periodic).
 * ---------------------------------------------------------------------- */
static const int A_fcc[4][3] = {{0, 0, 0}, {0, 2, 2}, {2, 0, 2}, {2, 2, 0}};
static const int B_basis[4][3] = {{0, 0, 0}, {0, 1, 1}, {1, 0, 1}, {1, 1, 0}};
static const int PAIR[6][2] = {{0, 1}, {0, 2}, {0, 3}, {1, 2}, {1, 3}, {2, 3}};

void orc_site_position(int L, int64_t i, int pos[3])
{
    int mu = (int)(i & 3), f = (int)((i >> 2) & 3);
    int64_t c = i >> 4;
    int x = (int)(c % L), y = (int)((c / L) % L), z = (int)(c / ((int64_t)L * L));
    pos[0] = 4 * x + A_fcc[f][0] + B_basis[mu][0];
    pos[1] = 4 * y + A_fcc[f][1] + B_basis[mu][1];
    pos[2] = 4 * z + A_fcc[f][2] + B_basis[mu][2];
}

/* nn[6*i + q]: the six sites at squared distance 2 (quarter units) from
 * site i under periodic wrap mod 4L, in increasing index order.
 * Returns 0, or -1 if some site does not have exactly six. */
int orc_build_nn(int L, int32_t *nn)
{
    int64_t N = 16LL * L * L * L;
    int64_t W = 4LL * L;
    int32_t *grid = (int32_t *)malloc((size_t)(W * W * W) * sizeof(int32_t));
    if (!grid) return -2;
    for (int64_t g = 0; g < W * W * W; ++g) grid[g] = -1;
    for (int64_t i = 0; i < N; ++i) {
        int p[3];
        orc_site_position(L, i, p);
        grid[p[0] + W * (p[1] + W * p[2])] = (int32_t)i;
    }
    int rc = 0;
    for (int64_t i = 0; i < N && rc == 0; ++i) {
        int p[3];
        orc_site_position(L, i, p);
        int cnt = 0;
        int32_t found[12];
        for (int dx = -1; dx <= 1; ++dx)
            for (int dy = -1; dy <= 1; ++dy)
                for (int dz = -1; dz <= 1; ++dz) {
                    if (dx * dx + dy * dy + dz * dz != 2) continue;
                    int64_t qx = ((p[0] + dx) % W + W) % W;
                    int64_t qy = ((p[1] + dy) % W + W) % W;
                    int64_t qz = ((p[2] + dz) % W + W) % W;
                    int32_t j = grid[qx + W * (qy + W * qz)];
                    if (j >= 0) found[cnt++] = j;
                }
        if (cnt != 6) { rc = -1; break; }
        /* insertion sort: increasing index */
        for (int a = 1; a < 6; ++a)
            for (int b = a; b > 0 && found[b - 1] > found[b]; --b) {
                int32_t t = found[b]; found[b] = found[b - 1]; found[b - 1] = t;
            }
        memcpy(nn + 6 * i, found, 6 * sizeof(int32_t));
    }
    free(grid);
    return rc;
}

static int is_nn(const int32_t *nn, int64_t i, int32_t j)
{
    for (int q = 0; q < 6; ++q)
        if (nn[6 * i + q] == j) return 1;
    return 0;
}

/* Bonds grouped by tetrahedron.  Bond b = 12 r + k.
 *   up tetrahedron of FCC point r: the four sites 4r + mu (same FCC point);
 *   down tetrahedron D(r): site 4r (basis 0) and its three neighbours that
 *   are not in its up tetrahedron, one of each basis 1, 2, 3.
 * Vertex v of a tetrahedron is its site of basis v; bond k pairs vertices
 * PAIR[k mod 6].  Returns 0, or -1 if the geometry does not close. */
int orc_build_bonds(int L, const int32_t *nn, int32_t *bond_i, int32_t *bond_j)
{
    int64_t N = 16LL * L * L * L;
    int64_t R = N / 4;
    for (int64_t r = 0; r < R; ++r) {
        int32_t up[4], down[4];
        for (int v = 0; v < 4; ++v) { up[v] = (int32_t)(4 * r + v); down[v] = -1; }
        down[0] = (int32_t)(4 * r);
        for (int q = 0; q < 6; ++q) {
            int32_t j = nn[6 * (4 * r) + q];
            if ((j >> 2) == r) continue; /* same FCC point: up tetrahedron */
            int v = j & 3;
            if (v == 0 || down[v] != -1) return -1;
            down[v] = j;
        }
        for (int v = 0; v < 4; ++v)
            if (down[v] < 0) return -1;
        for (int k = 0; k < 6; ++k) {
            int a = PAIR[k][0], b = PAIR[k][1];
            if (!is_nn(nn, up[a], up[b]) || !is_nn(nn, down[a], down[b])) return -1;
            bond_i[12 * r + k] = up[a];
            bond_j[12 * r + k] = up[b];
            bond_i[12 * r + 6 + k] = down[a];
            bond_j[12 * r + 6 + k] = down[b];
        }
    }
    return 0;
}

/* ------------------------------------------------------------------------
 * Sequential union-find.  Linking always puts the larger root under the
 * smaller one, so the root of a cluster is its minimum site index (the
 * canonical label).
 * ---------------------------------------------------------------------- */
static int32_t uf_find(int32_t *parent, int32_t x)
{
    int32_t root = x;
    while (parent[root] != root) root = parent[root];
    while (parent[x] != root) { int32_t nx = parent[x]; parent[x] = root; x = nx; }
    return root;
}

static void uf_union(int32_t *parent, int32_t a, int32_t b)
{
    int32_t ra = uf_find(parent, a), rb = uf_find(parent, b);
    if (ra == rb) return;
    if (ra < rb) parent[rb] = ra; else parent[ra] = rb;
}

/* Generic connected components of an edge list restricted to active edges;
 * labels[i] = minimum vertex index of i's component. */
int orc_clusters(int64_t nsites, int64_t nbonds, const int32_t *bi, const int32_t *bj,
                 const uint8_t *active, int32_t *labels)
{
    for (int64_t i = 0; i < nsites; ++i) labels[i] = (int32_t)i;
    for (int64_t b = 0; b < nbonds; ++b)
        if (active[b]) uf_union(labels, bi[b], bj[b]);
    for (int64_t i = 0; i < nsites; ++i) labels[i] = uf_find(labels, (int32_t)i);
    return 0;
}

/* ------------------------------------------------------------------------
 * Neumaier (improved Kahan) compensated summation.
 * ---------------------------------------------------------------------- */
typedef struct { double s, c; } nsum;

static void nsum_add(nsum *a, double x)
{
    double t = a->s + x;
    if (fabs(a->s) >= fabs(x)) a->c += (a->s - t) + x;
    else a->c += (x - t) + a->s;
    a->s = t;
}

static double nsum_get(const nsum *a) { return a->s + a->c; }

/* ------------------------------------------------------------------------
 * State.
 * ---------------------------------------------------------------------- */
typedef struct orc {
    int L, model, ncomp;
    int64_t N, NB;
    uint64_t seed;
    double J;
    uint64_t sweep;
    int32_t *nn;            /* N x 6 */
    int32_t *bond_i, *bond_j; /* 3N */
    int8_t *sigma;          /* Ising spins +-1 */
    double *spin;           /* continuous spins, SoA: spin[k*N + i] */
    int32_t *label;         /* canonical labels of the last sweep */
    uint8_t *active;        /* active bonds of the last sweep */
    double *proj;           /* projections s_i . r of the last sweep */
    double axis[3];         /* axis of the last sweep */
    nsum acc[5];            /* E, E^2, m^2, m^4, |m| */
    uint64_t count;
} orc;

void orc_free(orc *h)
{
    if (!h) return;
    free(h->nn); free(h->bond_i); free(h->bond_j); free(h->sigma); free(h->spin);
    free(h->label); free(h->active); free(h->proj);
    free(h);
}

/* start: 0 = ordered (Ising all +1, continuous e_0), 1 = random.
 * Random Ising: sigma_i = -1 iff bit i of the INIT stream is 1.
 * Random continuous: site i draws orc_unit_vector with call_base = i << 8. */
orc *orc_new(int L, int model, uint64_t seed, int start, double J)
{
    if (L < 1 || model < 1 || model > 3) return NULL;
    orc *h = (orc *)calloc(1, sizeof(orc));
    if (!h) return NULL;
    h->L = L; h->model = model; h->ncomp = model; h->seed = seed; h->J = J;
    h->N = 16LL * L * L * L;
    h->NB = 3 * h->N;
    h->nn = (int32_t *)malloc((size_t)h->N * 6 * sizeof(int32_t));
    h->bond_i = (int32_t *)malloc((size_t)h->NB * sizeof(int32_t));
    h->bond_j = (int32_t *)malloc((size_t)h->NB * sizeof(int32_t));
    h->label = (int32_t *)malloc((size_t)h->N * sizeof(int32_t));
    h->active = (uint8_t *)calloc((size_t)h->NB, 1);
    if (model == ORC_ISING) h->sigma = (int8_t *)malloc((size_t)h->N);
    else {
        h->spin = (double *)malloc((size_t)h->N * h->ncomp * sizeof(double));
        h->proj = (double *)malloc((size_t)h->N * sizeof(double));
    }
    if (!h->nn || !h->bond_i || !h->bond_j || !h->label || !h->active ||
        (model == ORC_ISING ? !h->sigma : (!h->spin || !h->proj))) { orc_free(h); return NULL; }
    if (orc_build_nn(L, h->nn) != 0 || orc_build_bonds(L, h->nn, h->bond_i, h->bond_j) != 0) {
        orc_free(h); return NULL;
    }
    for (int64_t i = 0; i < h->N; ++i) h->label[i] = (int32_t)i;
    if (model == ORC_ISING) {
        for (int64_t i = 0; i < h->N; ++i) {
            int neg = start ? (int)stream_bit(seed, INIT_SWEEP_FIELD, TAG_INIT, (uint64_t)i) : 0;
            h->sigma[i] = neg ? -1 : 1;
        }
    } else {
        for (int64_t i = 0; i < h->N; ++i) {
            double r[3] = {1.0, 0.0, 0.0};
            if (start) orc_unit_vector(seed, INIT_SWEEP_FIELD, TAG_INIT, (uint64_t)i << 8, h->ncomp, r);
            for (int k = 0; k < h->ncomp; ++k) h->spin[k * h->N + i] = r[k];
        }
    }
    return h;
}

/* Instantaneous observables of the current configuration (Eq. 1, Eq. 2):
 * E = -J sum_bonds s_i . s_j; m = |sum_i s_i| / N; m2 = m*m; m4 = m2*m2. */
void orc_measure(const orc *h, double *E, double *m2, double *m4, double *Mvec)
{
    double m;
    if (h->model == ORC_ISING) {
        int64_t M = 0, anti = 0;
        for (int64_t i = 0; i < h->N; ++i) M += h->sigma[i];
        for (int64_t b = 0; b < h->NB; ++b)
            if (h->sigma[h->bond_i[b]] != h->sigma[h->bond_j[b]]) anti += 1;
        *E = -h->J * (double)(h->NB - 2 * anti);
        m = fabs((double)M) / (double)h->N;
        if (Mvec) { Mvec[0] = (double)M; Mvec[1] = 0.0; Mvec[2] = 0.0; }
    } else {
        int n = h->ncomp;
        double Mk[3] = {0.0, 0.0, 0.0};
        for (int k = 0; k < n; ++k)
            for (int64_t i = 0; i < h->N; ++i) Mk[k] += h->spin[k * h->N + i];
        double e = 0.0;
        for (int64_t b = 0; b < h->NB; ++b) {
            int64_t i = h->bond_i[b], j = h->bond_j[b];
            double d = h->spin[i] * h->spin[j];
            for (int k = 1; k < n; ++k) d += h->spin[k * h->N + i] * h->spin[k * h->N + j];
            e += d;
        }
        *E = -h->J * e;
        double msq = Mk[0] * Mk[0];
        for (int k = 1; k < n; ++k) msq += Mk[k] * Mk[k];
        m = sqrt(msq) / (double)h->N;
        if (Mvec) { Mvec[0] = Mk[0]; Mvec[1] = Mk[1]; Mvec[2] = Mk[2]; }
    }
    *m2 = m * m;
    *m4 = (*m2) * (*m2);
}

/* One Swendsen-Wang sweep (Sec. 2; SW multi-cluster update, Wolff
 * embedding for n > 1), then the per-sweep measurement (Eq. 2). */
static void sweep_once(orc *h, double beta, double *trace)
{
    const int64_t N = h->N, NB = h->NB;
    const uint32_t sw = (uint32_t)h->sweep;
    const int n = h->ncomp;

    /* 1. bond activation */
    if (h->model == ORC_ISING) {
        uint64_t thr = orc_threshold(beta, h->J);
        for (int64_t b = 0; b < NB; ++b) {
            int32_t i = h->bond_i[b], j = h->bond_j[b];
            int act = 0;
            if (h->sigma[i] == h->sigma[j]) {
                uint32_t w = orc_bond_word(h->seed, sw, orc_bond_rng_id((uint64_t)b));
                act = ((uint64_t)w < thr);
            }
            h->active[b] = (uint8_t)act;
        }
    } else {
        orc_unit_vector(h->seed, sw, TAG_AXIS, 0, n, h->axis);
        for (int64_t i = 0; i < N; ++i) {
            double p = h->spin[i] * h->axis[0];
            for (int k = 1; k < n; ++k) p = p + h->spin[k * N + i] * h->axis[k];
            h->proj[i] = p;
        }
        double K2 = 2.0 * beta * h->J;
        for (int64_t b = 0; b < NB; ++b) {
            double x = h->proj[h->bond_i[b]] * h->proj[h->bond_j[b]];
            int act = 0;
            if (x > 0.0) {
                double prob = -expm1(-(K2 * x));
                uint32_t w = orc_bond_word(h->seed, sw, orc_bond_rng_id((uint64_t)b));
                act = ((uint64_t)w < prob_threshold(prob));
            }
            h->active[b] = (uint8_t)act;
        }
    }

    /* 2. clusters: canonical label = minimum site index */
    orc_clusters(N, NB, h->bond_i, h->bond_j, h->active, h->label);

    /* 3-4. each cluster flips with probability 1/2, keyed by its root */
    for (int64_t i = 0; i < N; ++i) {
        if (!stream_bit(h->seed, sw, TAG_FLIP, (uint64_t)h->label[i])) continue;
        if (h->model == ORC_ISING) {
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
    orc_measure(h, &E, &m2, &m4, Mv);
    nsum_add(&h->acc[0], E);
    nsum_add(&h->acc[1], E * E);
    nsum_add(&h->acc[2], m2);
    nsum_add(&h->acc[3], m4);
    nsum_add(&h->acc[4], sqrt(m2));
    h->count += 1;
    if (trace) { trace[0] = E; trace[1] = m2; trace[2] = m4; trace[3] = Mv[0]; }
    h->sweep += 1;
}

/* n sweeps at inverse temperature beta.  If trace is not NULL it receives
 * four doubles per sweep: E, m2, m4, M_x (Ising: M). */
int orc_sweep(orc *h, double beta, int64_t n, double *trace)
{
    if (!h || n < 0 || !(beta >= 0.0)) return -1;
    for (int64_t s = 0; s < n; ++s) sweep_once(h, beta, trace ? trace + 4 * s : NULL);
    return 0;
}

/* Accumulated sums since the last reset: out = {count, sum E, sum E^2,
 * sum m^2, sum m^4, sum |m|}. */
void orc_stats(const orc *h, double out[6])
{
    out[0] = (double)h->count;
    for (int k = 0; k < 5; ++k) out[k + 1] = nsum_get(&h->acc[k]);
}

void orc_reset_stats(orc *h)
{
    memset(h->acc, 0, sizeof(h->acc));
    h->count = 0;
}

int64_t orc_num_sites(const orc *h) { return h->N; }
uint64_t orc_get_sweep(const orc *h) { return h->sweep; }
void orc_set_sweep(orc *h, uint64_t s) { h->sweep = s; }
void orc_get_axis(const orc *h, double out[3]) { memcpy(out, h->axis, sizeof(h->axis)); }
void orc_get_labels(const orc *h, int32_t *out) { memcpy(out, h->label, (size_t)h->N * sizeof(int32_t)); }
void orc_get_active(const orc *h, uint8_t *out) { memcpy(out, h->active, (size_t)h->NB); }
void orc_get_nn(const orc *h, int32_t *out) { memcpy(out, h->nn, (size_t)h->N * 6 * sizeof(int32_t)); }

void orc_get_bonds(const orc *h, int32_t *bi, int32_t *bj)
{
    memcpy(bi, h->bond_i, (size_t)h->NB * sizeof(int32_t));
    memcpy(bj, h->bond_j, (size_t)h->NB * sizeof(int32_t));
}

/* Spins in canonical site order: Ising as int8 +-1 (N bytes); n > 1 as
 * doubles, site-major (N x n). */
void orc_get_spins(const orc *h, void *out)
{
    if (h->model == ORC_ISING) { memcpy(out, h->sigma, (size_t)h->N); return; }
    double *o = (double *)out;
    for (int64_t i = 0; i < h->N; ++i)
        for (int k = 0; k < h->ncomp; ++k) o[i * h->ncomp + k] = h->spin[k * h->N + i];
}

void orc_set_spins(orc *h, const void *in)
{
    if (h->model == ORC_ISING) { memcpy(h->sigma, in, (size_t)h->N); return; }
    const double *s = (const double *)in;
    for (int64_t i = 0; i < h->N; ++i)
        for (int k = 0; k < h->ncomp; ++k) h->spin[k * h->N + i] = s[i * h->ncomp + k];
}
