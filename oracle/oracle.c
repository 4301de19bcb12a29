/*
 * CPU oracle (test infrastructure only; never part of the product path).
 *
 * Plain, slow, obviously-correct FP64 reference for what the GPU path computes:
 *   - the state vector psi = C|0> of a circuit, applying gates one by one
 *     (definition of the amplitudes <b|C|0>, paper Sec. I eq. for |psi>);
 *   - sliced amplitudes: fixing a sliced tensor leg (qubit q between two gates) to
 *     value v is the projector |v><v| inserted on that wire at that point
 *     (Appendix B: the slicing delta acts on the wire as a projection);
 *   - psi_X = C2 Pi_X C1 |0> for a set X of partial-slice values (Sec. I.A,
 *     |psi_X> = sum_{i in X} |psi_i>, |psi_i> = sum_j C2|ji><ji|C1|0>);
 *   - marginals of a state on a subset of qubits (R[i] = ||psi_i||^2, Sec. I.A);
 *   - Philox4x32-10 (Salmon et al., SC'11) and the modified frugal rejection
 *     sampler of Sec. II.A in a fixed floating-point operation order.
 *
 * Conventions: bit q of a state index is qubit q.  A two-qubit gate on (q0, q1)
 * uses basis index 2*bit(q0) + bit(q1).  Compiled with -ffp-contract=off so that
 * every product and sum is rounded separately.
 *
 * Only tests/, the package's smoke entry and bench.py's CPU-baseline leg load this.
 */
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#include <math.h>

typedef struct { double re, im; } cd;

static inline cd cmul(cd a, cd b) {
    cd r;
    r.re = a.re * b.re - a.im * b.im;
    r.im = a.re * b.im + a.im * b.re;
    return r;
}
static inline cd cadd(cd a, cd b) { cd r; r.re = a.re + b.re; r.im = a.im + b.im; return r; }

/* ------------------------------------------------------------------ circuit */

typedef struct {
    int arity;
    int q[2];
    const cd *m;   /* (2^arity)^2 entries, row-major */
} ogate;

typedef struct {
    int n;
    int ng;
    ogate *g;
} ocirc;

/* Parse the serialized gate list (see the input module's docstring).  Returns 0 on
 * success.  The matrices point into buf, which must outlive the circuit. */
static int parse(const unsigned char *buf, size_t len, ocirc *c) {
    if (len < 12 || memcmp(buf, "RQC1", 4) != 0) return -1;
    uint32_t n, ng;
    memcpy(&n, buf + 4, 4);
    memcpy(&ng, buf + 8, 4);
    if (n == 0 || n > 40) return -1;
    c->n = (int)n;
    c->ng = (int)ng;
    c->g = (ogate *)calloc(ng ? ng : 1, sizeof(ogate));
    size_t off = 12;
    for (uint32_t i = 0; i < ng; i++) {
        uint32_t h[3];
        if (off + 12 > len) { free(c->g); return -1; }
        memcpy(h, buf + off, 12);
        off += 12;
        if (h[0] != 1 && h[0] != 2) { free(c->g); return -1; }
        size_t d = (size_t)1 << h[0];
        if (off + 16 * d * d > len) { free(c->g); return -1; }
        c->g[i].arity = (int)h[0];
        c->g[i].q[0] = (int)h[1];
        c->g[i].q[1] = h[0] == 2 ? (int)h[2] : -1;
        if (h[1] >= n || (h[0] == 2 && (h[2] >= n || h[2] == h[1]))) { free(c->g); return -1; }
        c->g[i].m = (const cd *)(buf + off);
        off += 16 * d * d;
    }
    return 0;
}

/* --------------------------------------------------------------- primitives */

void orc_zero_state(cd *psi, int n) {
    size_t N = (size_t)1 << n;
#pragma omp parallel for schedule(static)
    for (size_t i = 0; i < N; i++) { psi[i].re = 0.0; psi[i].im = 0.0; }
    psi[0].re = 1.0;
}

void orc_apply_1q(cd *psi, int n, int q, const cd *U) {
    size_t N = (size_t)1 << n, bit = (size_t)1 << q;
#pragma omp parallel for schedule(static)
    for (size_t i = 0; i < N; i++) {
        if (i & bit) continue;
        cd a = psi[i], b = psi[i | bit];
        psi[i] = cadd(cmul(U[0], a), cmul(U[1], b));
        psi[i | bit] = cadd(cmul(U[2], a), cmul(U[3], b));
    }
}

void orc_apply_2q(cd *psi, int n, int q0, int q1, const cd *U) {
    size_t N = (size_t)1 << n, b0 = (size_t)1 << q0, b1 = (size_t)1 << q1;
#pragma omp parallel for schedule(static)
    for (size_t i = 0; i < N; i++) {
        if ((i & b0) || (i & b1)) continue;
        size_t idx[4] = {i, i | b1, i | b0, i | b0 | b1};  /* basis 2*bit(q0)+bit(q1) */
        cd v[4], w[4];
        for (int r = 0; r < 4; r++) v[r] = psi[idx[r]];
        for (int r = 0; r < 4; r++) {
            cd acc = {0.0, 0.0};
            for (int s = 0; s < 4; s++) acc = cadd(acc, cmul(U[4 * r + s], v[s]));
            w[r] = acc;
        }
        for (int r = 0; r < 4; r++) psi[idx[r]] = w[r];
    }
}

/* |v><v| on qubit q: zero every component whose bit q differs from v. */
void orc_project(cd *psi, int n, int q, int v) {
    size_t N = (size_t)1 << n, bit = (size_t)1 << q;
#pragma omp parallel for schedule(static)
    for (size_t i = 0; i < N; i++) {
        int b = (i & bit) ? 1 : 0;
        if (b != v) { psi[i].re = 0.0; psi[i].im = 0.0; }
    }
}

static void apply_gate(cd *psi, int n, const ogate *g) {
    if (g->arity == 1) orc_apply_1q(psi, n, g->q[0], g->m);
    else orc_apply_2q(psi, n, g->q[0], g->q[1], g->m);
}

/* ------------------------------------------------------------- simulations */

/*
 * psi = C|0> with projectors.  Projector p fixes wire segment (proj_q[p], proj_s[p])
 * to proj_v[p]: segment s of qubit q is the wire just before the (s+1)-th two-qubit
 * gate acting on q (after all single-qubit gates preceding it); s equal to the number
 * of two-qubit gates on q denotes the circuit output of q.  Returns 0, or -1 on a bad
 * circuit / segment.
 */
int orc_simulate(const unsigned char *buf, size_t len, int n_proj, const int *proj_q,
                 const int *proj_s, const int *proj_v, cd *psi) {
    ocirc c;
    if (parse(buf, len, &c)) return -1;
    int n = c.n;
    int *cnt = (int *)calloc((size_t)n, sizeof(int));
    int *tot = (int *)calloc((size_t)n, sizeof(int));
    for (int i = 0; i < c.ng; i++)
        if (c.g[i].arity == 2) { tot[c.g[i].q[0]]++; tot[c.g[i].q[1]]++; }
    for (int p = 0; p < n_proj; p++)
        if (proj_q[p] < 0 || proj_q[p] >= n || proj_s[p] < 0 || proj_s[p] > tot[proj_q[p]] ||
            (proj_v[p] != 0 && proj_v[p] != 1)) {
            free(cnt); free(tot); free(c.g); return -1;
        }
    orc_zero_state(psi, n);
    for (int i = 0; i < c.ng; i++) {
        const ogate *g = &c.g[i];
        if (g->arity == 2) {
            for (int w = 0; w < 2; w++) {
                int q = g->q[w];
                for (int p = 0; p < n_proj; p++)
                    if (proj_q[p] == q && proj_s[p] == cnt[q]) orc_project(psi, n, q, proj_v[p]);
            }
            cnt[g->q[0]]++;
            cnt[g->q[1]]++;
        }
        apply_gate(psi, n, g);
    }
    for (int p = 0; p < n_proj; p++)
        if (proj_s[p] == tot[proj_q[p]]) orc_project(psi, n, proj_q[p], proj_v[p]);
    free(cnt); free(tot); free(c.g);
    return 0;
}

/*
 * psi = C2 D C1 |0>: the gates with in_c1[g] != 0 (a causally closed prefix set),
 * then the diagonal operator D = sum_{i in X} |i><i| on the k qubits s_qubits
 * (bit t of i is qubit s_qubits[t]; x_mask[i] != 0 marks i in X), then the other
 * gates in circuit order.  With D = identity this is C|0>.
 */
int orc_simulate_split(const unsigned char *buf, size_t len, const unsigned char *in_c1,
                       int k, const int *s_qubits, const unsigned char *x_mask, cd *psi) {
    ocirc c;
    if (parse(buf, len, &c)) return -1;
    int n = c.n;
    orc_zero_state(psi, n);
    for (int i = 0; i < c.ng; i++)
        if (in_c1[i]) apply_gate(psi, n, &c.g[i]);
    size_t N = (size_t)1 << n;
#pragma omp parallel for schedule(static)
    for (size_t idx = 0; idx < N; idx++) {
        size_t key = 0;
        for (int t = 0; t < k; t++) key |= ((idx >> s_qubits[t]) & 1u) << t;
        if (!x_mask[key]) { psi[idx].re = 0.0; psi[idx].im = 0.0; }
    }
    for (int i = 0; i < c.ng; i++)
        if (!in_c1[i]) apply_gate(psi, n, &c.g[i]);
    free(c.g);
    return 0;
}

/* Apply only the gates with sel[g] != 0, in circuit order, to |0>. */
int orc_simulate_subset(const unsigned char *buf, size_t len, const unsigned char *sel, cd *psi) {
    ocirc c;
    if (parse(buf, len, &c)) return -1;
    orc_zero_state(psi, c.n);
    for (int i = 0; i < c.ng; i++)
        if (sel[i]) apply_gate(psi, c.n, &c.g[i]);
    free(c.g);
    return 0;
}

/* out[i] = sum over basis states whose bits on qubits[0..k) read i of |psi|^2. */
void orc_marginal(const cd *psi, int n, int k, const int *qubits, double *out) {
    size_t N = (size_t)1 << n, K = (size_t)1 << k;
    for (size_t i = 0; i < K; i++) out[i] = 0.0;
    for (size_t idx = 0; idx < N; idx++) {
        size_t key = 0;
        for (int t = 0; t < k; t++) key |= ((idx >> qubits[t]) & 1u) << t;
        out[key] += psi[idx].re * psi[idx].re + psi[idx].im * psi[idx].im;
    }
}

/* ---------------------------------------------------------- Philox4x32-10 */
/* Salmon, Moraes, Dror, Shaw, "Parallel random numbers: as easy as 1, 2, 3", SC'11. */

static inline void mulhilo32(uint32_t a, uint32_t b, uint32_t *hi, uint32_t *lo) {
    uint64_t p = (uint64_t)a * (uint64_t)b;
    *hi = (uint32_t)(p >> 32);
    *lo = (uint32_t)p;
}

void orc_philox4x32_10(const uint32_t ctr_in[4], const uint32_t key_in[2], uint32_t out[4]) {
    uint32_t c0 = ctr_in[0], c1 = ctr_in[1], c2 = ctr_in[2], c3 = ctr_in[3];
    uint32_t k0 = key_in[0], k1 = key_in[1];
    for (int r = 0; r < 10; r++) {
        if (r > 0) { k0 += 0x9E3779B9u; k1 += 0xBB67AE85u; }
        uint32_t hi0, lo0, hi1, lo1;
        mulhilo32(0xD2511F53u, c0, &hi0, &lo0);
        mulhilo32(0xCD9E8D57u, c2, &hi1, &lo1);
        uint32_t n0 = hi1 ^ c1 ^ k0, n1 = lo1, n2 = hi0 ^ c3 ^ k1, n3 = lo0;
        c0 = n0; c1 = n1; c2 = n2; c3 = n3;
    }
    out[0] = c0; out[1] = c1; out[2] = c2; out[3] = c3;
}

/* -------------------------------------------------- rejection sampler (II.A) */

/*
 * Draws of step t use Philox4x32-10 with key (seed_lo, seed_hi) and counter
 * (t_lo, t_hi, stream, 0).  Stream 0: words 0,1 form the 64-bit batch draw (its low
 * b_bits bits are j); words 2,3 form u.  Stream 1: words 0,1 form v.  A 64-bit word w
 * becomes the double (w >> 11) * 2^-53 in [0, 1).
 */
static double u53(uint32_t lo, uint32_t hi) {
    uint64_t w = ((uint64_t)hi << 32) | lo;
    return (double)(w >> 11) * (1.0 / 9007199254740992.0);
}

void orc_draw(uint64_t seed, uint64_t t, uint64_t *jraw, double *u, double *v) {
    uint32_t key[2] = {(uint32_t)seed, (uint32_t)(seed >> 32)};
    uint32_t ctr[4] = {(uint32_t)t, (uint32_t)(t >> 32), 0u, 0u};
    uint32_t o[4];
    orc_philox4x32_10(ctr, key, o);
    *jraw = ((uint64_t)o[1] << 32) | o[0];
    *u = u53(o[2], o[3]);
    ctr[2] = 1u;
    orc_philox4x32_10(ctr, key, o);
    *v = u53(o[0], o[1]);
}

/*
 * One step of the modified frugal rejection sampler for each batch t in [0, T):
 * p[t*64 + i] = p_{i,j_t} (N_A = 64, i.e. 6 open qubits), batch index t0 + t.
 * The batch total p_j and the prefix sums follow a 32-lane Kogge-Stone scan of pair
 * sums s_l = p_{2l} + p_{2l+1}: offsets 1,2,4,8,16, x_l <- x_{l-off} + x_l.
 * p_j = x_31.  Accept iff u*alpha < p_j*N_B.  The prefix of element 2l is
 * x_{l-1} + p_{2l} (x_{-1} = 0), of element 2l+1 it is x_l; the pick is the smallest
 * i whose prefix exceeds tau = v*p_j, else the last i with p_i > 0.
 * accept[t] in {0,1}; pick[t] = i (valid when accepted).
 */
void orc_sample_batches(const double *p, int64_t T, int b_bits, double alpha, uint64_t seed,
                        uint64_t t0, unsigned char *accept, int32_t *pick) {
    double NB = ldexp(1.0, b_bits);
    for (int64_t t = 0; t < T; t++) {
        const double *pb = p + 64 * t;
        double x[32], s[32];
        for (int l = 0; l < 32; l++) { s[l] = pb[2 * l] + pb[2 * l + 1]; x[l] = s[l]; }
        for (int off = 1; off < 32; off <<= 1) {
            double y[32];
            for (int l = 0; l < 32; l++) y[l] = x[l];
            for (int l = off; l < 32; l++) x[l] = y[l - off] + y[l];
        }
        double pj = x[31];
        uint64_t jraw; double u, v;
        orc_draw(seed, t0 + (uint64_t)t, &jraw, &u, &v);
        double lhs = u * alpha, rhs = pj * NB;
        accept[t] = lhs < rhs ? 1 : 0;
        double tau = v * pj;
        int found = -1;
        for (int l = 0; l < 32 && found < 0; l++) {
            double excl = l == 0 ? 0.0 : x[l - 1];
            double c0 = excl + pb[2 * l];
            double c1 = x[l];
            if (c0 > tau) found = 2 * l;
            else if (c1 > tau) found = 2 * l + 1;
        }
        if (found < 0) {
            for (int i = 63; i >= 0; i--) if (pb[i] > 0.0) { found = i; break; }
            if (found < 0) found = 63;
        }
        pick[t] = found;
    }
}
