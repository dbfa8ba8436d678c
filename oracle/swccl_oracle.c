/*
 * swccl_oracle.c -- serial CPU oracle for the Swendsen-Wang sweep and for
 * connected-component labeling of bond configurations on L x L / H x W grids.
 *
 * TEST INFRASTRUCTURE ONLY.  Nothing in the product path may call, link or
 * load this file.  It shares no code with the CUDA library: its Philox,
 * threshold, activation, labeling, flip and observables are written here from
 * the published definitions, plainly and without any blocking or fusion.
 *
 * Source of each step (Weigel, "Connected component identification and
 * cluster update on GPU", arXiv:1105.5804):
 *   - Potts Hamiltonian H = -J sum_<ij> delta(s_i,s_j)          Sec. II, Eq. 1
 *   - bond probability p = 1 - exp(-beta J) (delta convention)   Sec. II, Eqs. 2-4
 *   - the three SW steps (activate, identify, re-spin)          Sec. II (enumerated list)
 *   - re-spin: one new state per cluster, read at its root       Sec. II.D
 *   - bond rule n_ij = 1 iff s_i = s_j and r < p                Sec. II.A, Eq. 7
 *   - labeling by breadth-first search, seeding every unlabeled
 *     site in site order, label = seed site                      Sec. II.B.1
 *   - periodic boundary conditions on the square lattice        Sec. II (end of intro)
 * The generator is Philox4x32-10 (Salmon, Moraes, Dror, Shaw, "Parallel
 * random numbers: as easy as 1, 2, 3", SC'11): 10 rounds, multipliers
 * 0xD2511F53 / 0xCD9E8D57, Weyl key increments 0x9E3779B9 / 0xBB67AE85.
 *
 * Conventions fixed where the paper is silent (each one is restated in the
 * design notes of the repository):
 *   - site index i = y*W + x; "east" = (x+1, y), "north" = (x, y+1)
 *   - packed bond mask: byte i>>2 holds site i in bits 2*(i&3) (east bond)
 *     and 2*(i&3)+1 (north bond)
 *   - Philox key = (seed_lo32, seed_hi32);
 *     counter = (c0, sweep_lo32, sweep_hi32, tag)
 *       tag 0 BOND: c0 = i>>1, word 2*(i&1)+dir (dir 0 east, 1 north)
 *       tag 1 FLIP: c0 = root site index, word 0
 *       tag 2 INIT: c0 = i, word 0, sweep 0
 *       tag 3 PERC: key = (k, 0), sweep 0, word mapping as BOND
 *       tag 4 SEED: c0 = seed block index (few-cluster update), words 0, 1
 *       tag 5 BOND3: simple-cubic lattice, c0 = i, word = dir
 *                    (0 = +x, 1 = +y, 2 = +z)
 *   - a bond between equal spins is open iff (uint64)r < T,
 *     T = min(2^32, floor(p * 2^32))
 *   - new cluster state F_q(w) = floor(w * q / 2^32)
 *
 * The few-cluster update (Sec. III, variant (c) of the single-cluster
 * algorithm) is the SW decomposition followed by: one seed site per block of
 * an ell x ell block grid (block side B = L / ell; the paper's tiles), every
 * cluster holding a seed is selected, and each selected cluster flips with
 * probability p_flip.  Readings where the paper is silent:
 *   - seed of block b = by*ell + bx: SEED draw (b, sweep), x = bx*B + F_B(w0),
 *     y = by*B + F_B(w1)
 *   - the cluster with root R flips iff (uint64)w1 < P, w = FLIP draw of R,
 *     P = min(2^32, floor(p_flip * 2^32)); its new state is
 *     (s + 1 + F_{q-1}(w0)) mod q, a uniform choice among the other q - 1
 *     states (for q = 2: s -> 1 - s, the paper's flip)
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

enum { OR_TAG_BOND = 0, OR_TAG_FLIP = 1, OR_TAG_INIT = 2, OR_TAG_PERC = 3, OR_TAG_SEED = 4, OR_TAG_BOND3 = 5 };

/* ------------------------------------------------------------------------ */
/* Philox4x32-10, written from the SC'11 description.                        */
/* ------------------------------------------------------------------------ */
void or_philox4x32_10(const uint32_t ctr[4], const uint32_t key[2], uint32_t out[4])
{
    uint32_t c0 = ctr[0], c1 = ctr[1], c2 = ctr[2], c3 = ctr[3];
    uint32_t k0 = key[0], k1 = key[1];
    for (int round = 0; round < 10; round++) {
        if (round > 0) {               /* key schedule: Weyl sequence */
            k0 += 0x9E3779B9u;
            k1 += 0xBB67AE85u;
        }
        uint64_t prod0 = (uint64_t)0xD2511F53u * (uint64_t)c0;
        uint64_t prod1 = (uint64_t)0xCD9E8D57u * (uint64_t)c2;
        uint32_t hi0 = (uint32_t)(prod0 >> 32), lo0 = (uint32_t)prod0;
        uint32_t hi1 = (uint32_t)(prod1 >> 32), lo1 = (uint32_t)prod1;
        uint32_t n0 = hi1 ^ c1 ^ k0;
        uint32_t n1 = lo1;
        uint32_t n2 = hi0 ^ c3 ^ k1;
        uint32_t n3 = lo0;
        c0 = n0; c1 = n1; c2 = n2; c3 = n3;
    }
    out[0] = c0; out[1] = c1; out[2] = c2; out[3] = c3;
}

/* One 32-bit word of Philox output for (seed, c0, sweep, tag), word w. */
static uint32_t draw_word(uint64_t seed, uint32_t c0, uint64_t sweep, uint32_t tag, int w)
{
    uint32_t ctr[4] = { c0, (uint32_t)sweep, (uint32_t)(sweep >> 32), tag };
    uint32_t key[2] = { (uint32_t)seed, (uint32_t)(seed >> 32) };
    uint32_t out[4];
    or_philox4x32_10(ctr, key, out);
    return out[w];
}

/* ------------------------------------------------------------------------ */
/* Coupling and threshold (Sec. II, Eqs. 2-4: p = 1 - exp(-beta J)).         */
/* ------------------------------------------------------------------------ */
/* convention: 1 = Potts delta coupling (K = beta J),
 *             2 = Ising +-1 spins (H = -J sum sigma sigma, K = 2 beta J),
 *             0 = automatic: Ising for q = 2, Potts delta otherwise. */
double or_coupling_K(int q, double beta, double J, int convention)
{
    if (convention == 0) convention = (q == 2) ? 2 : 1;
    return (convention == 2) ? 2.0 * beta * J : beta * J;
}

/* T = min(2^32, floor(p 2^32)), p = -expm1(-K), in IEEE double. */
uint64_t or_threshold(double K)
{
    if (!(K > 0.0)) return 0;
    double p = -expm1(-K);
    double t = floor(p * 4294967296.0);
    if (t >= 4294967296.0) return (uint64_t)1 << 32;
    if (t < 0.0) return 0;
    return (uint64_t)t;
}

/* New cluster state from a 32-bit word: floor(w q / 2^32). */
int or_flip_state(uint32_t w, int q)
{
    return (int)(((uint64_t)w * (uint64_t)q) >> 32);
}

/* ------------------------------------------------------------------------ */
/* Mask helpers (packed, 2 bits per site).                                   */
/* ------------------------------------------------------------------------ */
static int bond_open(const uint8_t* mask, int64_t i, int dir)
{
    return (mask[i >> 2] >> (2 * (i & 3) + dir)) & 1;
}

static void set_bond(uint8_t* mask, int64_t i, int dir)
{
    mask[i >> 2] |= (uint8_t)(1u << (2 * (i & 3) + dir));
}

int64_t or_mask_bytes(int64_t n_sites) { return (n_sites + 3) / 4; }

/* ------------------------------------------------------------------------ */
/* Initial spins: cold start all s = 0, hot start s_i = F_q(INIT draw).      */
/* ------------------------------------------------------------------------ */
void or_init_spins(int L, int q, uint64_t seed, int hot, int8_t* spins)
{
    int64_t N = (int64_t)L * L;
    for (int64_t i = 0; i < N; i++) {
        if (hot)
            spins[i] = (int8_t)or_flip_state(draw_word(seed, (uint32_t)i, 0, OR_TAG_INIT, 0), q);
        else
            spins[i] = 0;
    }
}

/* ------------------------------------------------------------------------ */
/* Step 1: bond activation on the periodic L x L lattice (Sec. II.A).        */
/* n_ij = 1 iff s_i = s_j and r_ij < p, r_ij from the BOND draw.             */
/* ------------------------------------------------------------------------ */
void or_activate(int L, const int8_t* spins, uint64_t seed, uint64_t sweep, uint64_t T,
                 uint8_t* mask)
{
    int64_t N = (int64_t)L * L;
    memset(mask, 0, (size_t)or_mask_bytes(N));
    for (int y = 0; y < L; y++) {
        for (int x = 0; x < L; x++) {
            int64_t i = (int64_t)y * L + x;
            int64_t east = (int64_t)y * L + (x + 1) % L;
            int64_t north = (int64_t)((y + 1) % L) * L + x;
            int64_t nbr[2] = { east, north };
            for (int dir = 0; dir < 2; dir++) {
                if (spins[i] != spins[nbr[dir]]) continue;      /* n_ij = 0 */
                uint32_t r = draw_word(seed, (uint32_t)(i >> 1), sweep, OR_TAG_BOND,
                                       (int)(2 * (i & 1) + dir));
                if ((uint64_t)r < T) set_bond(mask, i, dir);
            }
        }
    }
}

/* Critical bond percolation (p = 1/2) mask for seed k on an H x W grid:
 * every one of the 2N bonds is open iff the PERC draw is < 2^31. */
void or_perc_mask(int H, int W, uint64_t k, uint8_t* mask)
{
    int64_t N = (int64_t)H * W;
    memset(mask, 0, (size_t)or_mask_bytes(N));
    for (int64_t i = 0; i < N; i++) {
        for (int dir = 0; dir < 2; dir++) {
            uint32_t r = draw_word(k, (uint32_t)(i >> 1), 0, OR_TAG_PERC, (int)(2 * (i & 1) + dir));
            if ((uint64_t)r < ((uint64_t)1 << 31)) set_bond(mask, i, dir);
        }
    }
}

/* Image segmentation bonds: a bond is open iff the two pixels have the same
 * level (Potts mapping of an image, Sec. I and II).  With periodic == 0 a
 * bond that would leave the grid is closed. */
void or_bonds_from_pixels(int H, int W, int periodic, const uint8_t* px, uint8_t* mask)
{
    int64_t N = (int64_t)H * W;
    memset(mask, 0, (size_t)or_mask_bytes(N));
    for (int y = 0; y < H; y++) {
        for (int x = 0; x < W; x++) {
            int64_t i = (int64_t)y * W + x;
            if (periodic || x + 1 < W) {
                int64_t e = (int64_t)y * W + (x + 1) % W;
                if (px[i] == px[e]) set_bond(mask, i, 0);
            }
            if (periodic || y + 1 < H) {
                int64_t n = (int64_t)((y + 1) % H) * W + x;
                if (px[i] == px[n]) set_bond(mask, i, 1);
            }
        }
    }
}

/* ------------------------------------------------------------------------ */
/* Step 2: cluster identification by breadth-first search (Sec. II.B.1).    */
/* Every site not yet labeled seeds a new cluster, in increasing site order; */
/* the whole cluster receives the seed's index.  The seed is therefore the   */
/* smallest index of its cluster.  Returns the number of clusters, or -1 on  */
/* allocation failure.                                                       */
/* ------------------------------------------------------------------------ */
int64_t or_label(int H, int W, int periodic, const uint8_t* mask, int32_t* labels)
{
    int64_t N = (int64_t)H * W;
    int64_t* queue = (int64_t*)malloc(sizeof(int64_t) * (size_t)(N > 0 ? N : 1));
    if (!queue) return -1;
    for (int64_t i = 0; i < N; i++) labels[i] = -1;
    int64_t n_clusters = 0;
    for (int64_t seed = 0; seed < N; seed++) {
        if (labels[seed] != -1) continue;
        n_clusters++;
        labels[seed] = (int32_t)seed;
        int64_t head = 0, tail = 0;
        queue[tail++] = seed;
        while (head < tail) {
            int64_t u = queue[head++];
            int y = (int)(u / W), x = (int)(u % W);
            /* the four lattice neighbours and the bond that joins each to u */
            int64_t v[4];
            int open[4];
            /* east: bond (u, east) is u's east bond */
            if (periodic || x + 1 < W) { v[0] = (int64_t)y * W + (x + 1) % W; open[0] = bond_open(mask, u, 0); }
            else { v[0] = -1; open[0] = 0; }
            /* north: bond (u, north) is u's north bond */
            if (periodic || y + 1 < H) { v[1] = (int64_t)((y + 1) % H) * W + x; open[1] = bond_open(mask, u, 1); }
            else { v[1] = -1; open[1] = 0; }
            /* west: bond (west, u) is the west site's east bond */
            if (periodic || x > 0) { v[2] = (int64_t)y * W + (x + W - 1) % W; open[2] = bond_open(mask, v[2], 0); }
            else { v[2] = -1; open[2] = 0; }
            /* south: bond (south, u) is the south site's north bond */
            if (periodic || y > 0) { v[3] = (int64_t)((y + H - 1) % H) * W + x; open[3] = bond_open(mask, v[3], 1); }
            else { v[3] = -1; open[3] = 0; }
            for (int k = 0; k < 4; k++) {
                if (!open[k] || labels[v[k]] != -1) continue;
                labels[v[k]] = (int32_t)seed;
                queue[tail++] = v[k];
            }
        }
    }
    free(queue);
    return n_clusters;
}

/* ------------------------------------------------------------------------ */
/* Step 3: every cluster takes a new state drawn at its root (Sec. II.D);    */
/* the root is the cluster's label, the draw is FLIP keyed by the root.      */
/* ------------------------------------------------------------------------ */
void or_flip(int64_t N, int q, uint64_t seed, uint64_t sweep, const int32_t* labels, int8_t* spins)
{
    for (int64_t i = 0; i < N; i++) {
        uint32_t root = (uint32_t)labels[i];
        spins[i] = (int8_t)or_flip_state(draw_word(seed, root, sweep, OR_TAG_FLIP, 0), q);
    }
}

/* Observables of a configuration (Eq. 1): out[0] = number of lattice bonds
 * joining equal spins, out[1 + k] = number of sites in state k. */
void or_observables(int L, int q, const int8_t* spins, int64_t* out)
{
    for (int k = 0; k <= q; k++) out[k] = 0;
    for (int y = 0; y < L; y++) {
        for (int x = 0; x < L; x++) {
            int64_t i = (int64_t)y * L + x;
            if (spins[i] == spins[(int64_t)y * L + (x + 1) % L]) out[0]++;
            if (spins[i] == spins[(int64_t)((y + 1) % L) * L + x]) out[0]++;
            out[1 + spins[i]]++;
        }
    }
}

/* One full SW sweep with index `sweep`: activate, identify, re-spin, then
 * measure.  mask / labels receive this sweep's bond mask and canonical
 * labels; spins are replaced by the new configuration.  Returns 0, or -1 on
 * allocation failure. */
int or_sweep(int L, int q, uint64_t T, uint64_t seed, uint64_t sweep, int8_t* spins,
             uint8_t* mask, int32_t* labels, int64_t* obs)
{
    int64_t N = (int64_t)L * L;
    or_activate(L, spins, seed, sweep, T, mask);
    if (or_label(L, L, 1, mask, labels) < 0) return -1;
    or_flip(N, q, seed, sweep, labels, spins);
    if (obs) or_observables(L, q, spins, obs);
    return 0;
}

/* n_sweeps consecutive sweeps starting at sweep0; obs receives (1+q) int64
 * per sweep.  Scratch is allocated here.  Returns 0, or -1 on failure. */
int or_chain(int L, int q, uint64_t T, uint64_t seed, uint64_t sweep0, int64_t n_sweeps,
             int8_t* spins, int64_t* obs)
{
    int64_t N = (int64_t)L * L;
    uint8_t* mask = (uint8_t*)malloc((size_t)or_mask_bytes(N));
    int32_t* labels = (int32_t*)malloc(sizeof(int32_t) * (size_t)N);
    if (!mask || !labels) { free(mask); free(labels); return -1; }
    int rc = 0;
    for (int64_t s = 0; s < n_sweeps && rc == 0; s++)
        rc = or_sweep(L, q, T, seed, sweep0 + (uint64_t)s, spins, mask, labels,
                      obs ? obs + s * (1 + q) : NULL);
    free(mask);
    free(labels);
    return rc;
}

/* ------------------------------------------------------------------------ */
/* Few-cluster update (Sec. III, variant (c)): SW bonds and clusters, then    */
/* only the clusters of one seed per block flip, each with probability P.    */
/* ------------------------------------------------------------------------ */
/* Seed site of block b (0 <= b < ell*ell) at this sweep. */
int64_t or_few_seed(int L, int ell, uint64_t seed, uint64_t sweep, int64_t b)
{
    int B = L / ell;
    int64_t by = b / ell, bx = b % ell;
    int64_t x = bx * B + or_flip_state(draw_word(seed, (uint32_t)b, sweep, OR_TAG_SEED, 0), B);
    int64_t y = by * B + or_flip_state(draw_word(seed, (uint32_t)b, sweep, OR_TAG_SEED, 1), B);
    return y * L + x;
}

/* spins updated in place; mask, labels as or_sweep.  Requires ell >= 1 and
 * L % ell == 0.  Returns 0, or -1 on failure. */
int or_few_sweep(int L, int q, uint64_t T, uint64_t P, int ell, uint64_t seed, uint64_t sweep, int8_t* spins,
                 uint8_t* mask, int32_t* labels, int64_t* obs)
{
    int64_t N = (int64_t)L * L;
    if (ell < 1 || L % ell != 0) return -1;
    or_activate(L, spins, seed, sweep, T, mask);
    if (or_label(L, L, 1, mask, labels) < 0) return -1;
    uint8_t* selected = (uint8_t*)calloc((size_t)N, 1);
    if (!selected) return -1;
    for (int64_t b = 0; b < (int64_t)ell * ell; b++)
        selected[labels[or_few_seed(L, ell, seed, sweep, b)]] = 1;
    for (int64_t i = 0; i < N; i++) {
        uint32_t root = (uint32_t)labels[i];
        if (!selected[root]) continue;
        uint32_t accept = draw_word(seed, root, sweep, OR_TAG_FLIP, 1);
        if ((uint64_t)accept >= P) continue;
        int shift = 1 + or_flip_state(draw_word(seed, root, sweep, OR_TAG_FLIP, 0), q - 1);
        spins[i] = (int8_t)((spins[i] + shift) % q);
    }
    free(selected);
    if (obs) or_observables(L, q, spins, obs);
    return 0;
}

int or_few_chain(int L, int q, uint64_t T, uint64_t P, int ell, uint64_t seed, uint64_t sweep0, int64_t n_sweeps,
                 int8_t* spins, int64_t* obs)
{
    int64_t N = (int64_t)L * L;
    uint8_t* mask = (uint8_t*)malloc((size_t)or_mask_bytes(N));
    int32_t* labels = (int32_t*)malloc(sizeof(int32_t) * (size_t)N);
    if (!mask || !labels) { free(mask); free(labels); return -1; }
    int rc = 0;
    for (int64_t s = 0; s < n_sweeps && rc == 0; s++)
        rc = or_few_sweep(L, q, T, P, ell, seed, sweep0 + (uint64_t)s, spins, mask, labels,
                          obs ? obs + s * (1 + q) : NULL);
    free(mask);
    free(labels);
    return rc;
}

/* ------------------------------------------------------------------------ */
/* Simple-cubic lattice (the generalisation the paper names in Secs. II and  */
/* II.B: the same three SW steps with six neighbours instead of four).       */
/* Box X x Y x Z, periodic; site i = (z*Y + y)*X + x; each site owns its      */
/* bonds to (x+1, y, z), (x, y+1, z), (x, y, z+1).  Bond mask: one byte per   */
/* site, bit d = bond in direction d (0 = +x, 1 = +y, 2 = +z).                */
/* ------------------------------------------------------------------------ */
static int64_t nb3(int X, int Y, int Z, int64_t i, int dir)
{
    int64_t x = i % X, y = (i / X) % Y, z = i / ((int64_t)X * Y);
    if (dir == 0) x = (x + 1) % X;
    else if (dir == 1) y = (y + 1) % Y;
    else z = (z + 1) % Z;
    return (z * Y + y) * X + x;
}

void or3_init_spins(int X, int Y, int Z, int q, uint64_t seed, int hot, int8_t* spins)
{
    int64_t N = (int64_t)X * Y * Z;
    for (int64_t i = 0; i < N; i++)
        spins[i] = hot ? (int8_t)or_flip_state(draw_word(seed, (uint32_t)i, 0, OR_TAG_INIT, 0), q) : 0;
}

/* Eq. 7 on the three bonds each site owns. */
void or3_activate(int X, int Y, int Z, const int8_t* spins, uint64_t seed, uint64_t sweep, uint64_t T,
                  uint8_t* mask)
{
    int64_t N = (int64_t)X * Y * Z;
    for (int64_t i = 0; i < N; i++) {
        mask[i] = 0;
        for (int dir = 0; dir < 3; dir++) {
            if (spins[i] != spins[nb3(X, Y, Z, i, dir)]) continue;
            uint32_t r = draw_word(seed, (uint32_t)i, sweep, OR_TAG_BOND3, dir);
            if ((uint64_t)r < T) mask[i] |= (uint8_t)(1u << dir);
        }
    }
}

/* Breadth-first search seeded in site order (Sec. II.B.1), six neighbours:
 * labels = smallest site index of the cluster.  Returns the number of
 * clusters, or -1 on allocation failure. */
int64_t or3_label(int X, int Y, int Z, const uint8_t* mask, int32_t* labels)
{
    int64_t N = (int64_t)X * Y * Z;
    int64_t* queue = (int64_t*)malloc(sizeof(int64_t) * (size_t)(N > 0 ? N : 1));
    if (!queue) return -1;
    for (int64_t i = 0; i < N; i++) labels[i] = -1;
    int64_t n_clusters = 0;
    for (int64_t seed = 0; seed < N; seed++) {
        if (labels[seed] != -1) continue;
        n_clusters++;
        labels[seed] = (int32_t)seed;
        int64_t head = 0, tail = 0;
        queue[tail++] = seed;
        while (head < tail) {
            int64_t u = queue[head++];
            int64_t x = u % X, y = (u / X) % Y, z = u / ((int64_t)X * Y);
            for (int dir = 0; dir < 3; dir++) {
                /* forward: u's own bond; backward: the bond the neighbour
                 * below in this direction owns */
                int64_t fwd = nb3(X, Y, Z, u, dir);
                int64_t bx = x, by = y, bz = z;
                if (dir == 0) bx = (x + X - 1) % X;
                else if (dir == 1) by = (y + Y - 1) % Y;
                else bz = (z + Z - 1) % Z;
                int64_t bwd = (bz * Y + by) * X + bx;
                if (((mask[u] >> dir) & 1) && labels[fwd] == -1) {
                    labels[fwd] = (int32_t)seed;
                    queue[tail++] = fwd;
                }
                if (((mask[bwd] >> dir) & 1) && labels[bwd] == -1) {
                    labels[bwd] = (int32_t)seed;
                    queue[tail++] = bwd;
                }
            }
        }
    }
    free(queue);
    return n_clusters;
}

/* n_eq over the 3N bonds, then sites per state. */
void or3_observables(int X, int Y, int Z, int q, const int8_t* spins, int64_t* out)
{
    int64_t N = (int64_t)X * Y * Z;
    for (int k = 0; k <= q; k++) out[k] = 0;
    for (int64_t i = 0; i < N; i++) {
        for (int dir = 0; dir < 3; dir++)
            if (spins[i] == spins[nb3(X, Y, Z, i, dir)]) out[0]++;
        out[1 + spins[i]]++;
    }
}

int or3_sweep(int X, int Y, int Z, int q, uint64_t T, uint64_t seed, uint64_t sweep, int8_t* spins,
              uint8_t* mask, int32_t* labels, int64_t* obs)
{
    int64_t N = (int64_t)X * Y * Z;
    or3_activate(X, Y, Z, spins, seed, sweep, T, mask);
    if (or3_label(X, Y, Z, mask, labels) < 0) return -1;
    or_flip(N, q, seed, sweep, labels, spins);
    if (obs) or3_observables(X, Y, Z, q, spins, obs);
    return 0;
}

int or3_chain(int X, int Y, int Z, int q, uint64_t T, uint64_t seed, uint64_t sweep0, int64_t n_sweeps,
              int8_t* spins, int64_t* obs)
{
    int64_t N = (int64_t)X * Y * Z;
    uint8_t* mask = (uint8_t*)malloc((size_t)N);
    int32_t* labels = (int32_t*)malloc(sizeof(int32_t) * (size_t)N);
    if (!mask || !labels) { free(mask); free(labels); return -1; }
    int rc = 0;
    for (int64_t s = 0; s < n_sweeps && rc == 0; s++)
        rc = or3_sweep(X, Y, Z, q, T, seed, sweep0 + (uint64_t)s, spins, mask, labels,
                       obs ? obs + s * (1 + q) : NULL);
    free(mask);
    free(labels);
    return rc;
}
