/*
 * ising_oracle.c -- the ORACLE for the replica-parallel Metropolis sweep with
 * parallel tempering (Dickson, Karimi & Hamze, "Importance of Explicit
 * Vectorization for CPU and GPU Software Performance", arXiv:1004.0024).
 *
 * TEST INFRASTRUCTURE ONLY.  This file is a plain, slow, obviously correct CPU
 * restatement of what the GPU path computes.  It shares no code, header,
 * table or constant generator with the CUDA library; only the tests, the
 * smoke check and bench.py's cpu_baseline / reference leg may call it.
 *
 * What it follows, step by step:
 *   - Ising cost function (paper section 1):
 *         f(s) = -sum_i h_i s_i - sum_{i,j} J_ij s_i s_j ,  s_i in {-1,+1}.
 *     Reading: every undirected edge is counted once in the pair sum.  This
 *     is the reading under which the field update of Figure 6,
 *     h_eff[target] -= 2*S_mul*J, keeps h_eff_i = h_i + sum_j J_ij s_j.
 *   - Metropolis sweep (Figure 1): visit spins i = 0..N-1 in index order;
 *     draw one uniform; if it is below the flip probability, flip s_i and
 *     update the data of every adjacent spin (Figure 6: f_j -= 2 s_i J_ij,
 *     with s_i the value before the flip).
 *     Readings: flip probability = min(1, exp(-beta dE)), dE = 2 s_i f_i.
 *     The uniform is a uint32 word u and the probability is the integer
 *     threshold T_beta(k) = floor(2^32 exp(-2 beta k)) built in FP64, so the
 *     test "uniform < probability" is u < T_beta(k) (strict, as in Figure 1),
 *     and k = s_i f_i <= 0 always flips.  One word is drawn per visit, also
 *     when the flip is certain.
 *   - MT19937 (paper ref [9], the generator of section 3 / Figure 8):
 *     Matsumoto & Nishimura's recurrence and tempering, seeded with their
 *     init_genrand.  One generator per replica, seeded with seed + r.
 *   - Parallel tempering (section 1 and section 3.1 mention it; the rule is in
 *     the paper's refs [16], [17], not in the paper).  Reading: standard
 *     replica exchange between adjacent inverse temperatures, label swaps
 *     (states stay in their slots), pass p tries the pairs (k, k+1) with
 *     k = p mod 2, ascending k, accept if d = E_lo - E_hi <= 0 or
 *     u < floor(2^32 exp(-(beta_{k+1} - beta_k) d)); one word per attempted
 *     pair from a per-instance swap stream (MT19937 seeded with seed + R).
 *   - Philox4x32-10 (Salmon, Moraes, Dror & Shaw, SC'11) as the alternative
 *     counter-based generator, with this counter map (spin i = t*S + q for a
 *     declared slice size S):
 *         sweep word  : key (seed, r),          ctr ((t>>2)*S + q, c, inst, 0), lane t&3
 *         init word   : key (seed, r),          ctr ((t>>2)*S + q, 0, inst, 3), lane t&3
 *         swap word   : key (seed, 0xFFFFFFFF), ctr (j>>2, p, inst, 1),       lane j&3
 *     where c counts the sweeps the instance has done, p the PT passes, and
 *     j = k>>1 is the ordinal of pair (k, k+1) within its pass.
 *   - Initial state: s_i = +1 when bit 31 of the i-th init word is set, else
 *     -1.  For MT19937 the init words are the first N outputs of the replica's
 *     stream, and sweep c uses outputs N(1+c) .. N(2+c)-1.  Slot r starts at
 *     temperature index r.
 *   - Split couplings (optional, orc_sim_set_trotter): the layered model of
 *     section 4 comes from a Trotter decomposition whose inter-slice coupling
 *     depends on the temperature.  Reading: temperature k weights a state by
 *     exp(-beta_k E_space - K_k C), E_space the cost function over the
 *     in-slice edges and C = -sum over the inter-slice (Trotter) pairs of
 *     s s'; a flip has z = 2 s (beta f_space + K tau), tau the sum of the
 *     spin's Trotter neighbours, and a swap z = dbeta dE + dK dC.  Each has
 *     the threshold T = min(floor(2^32 e^-z), 2^32 - 1), T = 2^32 - 1 for
 *     z <= 0, and is accepted iff T = 2^32 - 1 or u < T (so that one 32-bit
 *     table entry holds the whole decision).
 *
 * Replicas are independent between PT passes, so sweeps of different
 * replicas run on a pthread pool (one replica chunk per thread); the order of
 * work inside a replica is exactly the sequential order above.
 */
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#include <math.h>
#include <pthread.h>
#include <unistd.h>

/* ---------------------------------------------------------------- MT19937 */
/* Matsumoto & Nishimura (1998): degree n = 624, middle word m = 397,
 * twist matrix a = 0x9908B0DF, upper/lower split at bit 31, tempering
 * (u,d) = (11, 0xFFFFFFFF), (s,b) = (7, 0x9D2C5680), (t,c) = (15, 0xEFC60000),
 * l = 18.  Paper Figure 8 shows the two twist lines restated in regenerate(). */
typedef struct {
    uint32_t x[624];
    int next;
} orc_mt;

void orc_mt_seed(orc_mt* g, uint32_t seed)
{
    g->x[0] = seed;
    for (int i = 1; i < 624; i++) {
        uint32_t prev = g->x[i - 1];
        g->x[i] = 1812433253u * (prev ^ (prev >> 30)) + (uint32_t)i;
    }
    g->next = 624;
}

static void orc_mt_regenerate(orc_mt* g)
{
    for (int k = 0; k < 624; k++) {
        uint32_t y = (g->x[k] & 0x80000000u) | (g->x[(k + 1) % 624] & 0x7FFFFFFFu);
        uint32_t v = g->x[(k + 397) % 624] ^ (y >> 1);
        if (y & 1u)
            v ^= 0x9908B0DFu;
        g->x[k] = v;
    }
    g->next = 0;
}

uint32_t orc_mt_next(orc_mt* g)
{
    if (g->next >= 624)
        orc_mt_regenerate(g);
    uint32_t y = g->x[g->next++];
    y ^= (y >> 11);
    y ^= (y << 7) & 0x9D2C5680u;
    y ^= (y << 15) & 0xEFC60000u;
    y ^= (y >> 18);
    return y;
}

void orc_mt_stream(uint32_t seed, int64_t n, uint32_t* out)
{
    orc_mt g;
    orc_mt_seed(&g, seed);
    for (int64_t i = 0; i < n; i++)
        out[i] = orc_mt_next(&g);
}

/* ---------------------------------------------------------- Philox4x32-10 */
/* Salmon et al. (SC'11): 10 rounds; each round multiplies counter words 0 and
 * 2 by 0xD2511F53 and 0xCD9E8D57 (64-bit products split into hi/lo), then
 * out = (hi1 ^ c1 ^ k0, lo1, hi0 ^ c3 ^ k1, lo0); between rounds the key is
 * bumped by the Weyl constants (0x9E3779B9, 0xBB67AE85). */
void orc_philox(const uint32_t ctr[4], const uint32_t key[2], uint32_t out[4])
{
    uint32_t c0 = ctr[0], c1 = ctr[1], c2 = ctr[2], c3 = ctr[3];
    uint32_t k0 = key[0], k1 = key[1];
    for (int round = 0; round < 10; round++) {
        if (round > 0) {
            k0 += 0x9E3779B9u;
            k1 += 0xBB67AE85u;
        }
        uint64_t p0 = (uint64_t)0xD2511F53u * (uint64_t)c0;
        uint64_t p1 = (uint64_t)0xCD9E8D57u * (uint64_t)c2;
        uint32_t hi0 = (uint32_t)(p0 >> 32), lo0 = (uint32_t)p0;
        uint32_t hi1 = (uint32_t)(p1 >> 32), lo1 = (uint32_t)p1;
        uint32_t n0 = hi1 ^ c1 ^ k0;
        uint32_t n2 = hi0 ^ c3 ^ k1;
        c0 = n0;
        c1 = lo1;
        c2 = n2;
        c3 = lo0;
    }
    out[0] = c0;
    out[1] = c1;
    out[2] = c2;
    out[3] = c3;
}

/* One Philox word under the counter map described in the file header. */
static uint32_t philox_word(uint32_t k0, uint32_t k1, uint32_t c0, uint32_t c1,
                            uint32_t c2, uint32_t c3, int lane)
{
    uint32_t ctr[4] = {c0, c1, c2, c3};
    uint32_t key[2] = {k0, k1};
    uint32_t out[4];
    orc_philox(ctr, key, out);
    return out[lane];
}

/* ------------------------------------------------------------- thresholds */
/* T_beta(k) = floor(2^32 exp(-2 beta k)) for k >= 1, in FP64. */
uint32_t orc_flip_threshold(double beta, int64_t k)
{
    double p = exp(-2.0 * beta * (double)k);
    return (uint32_t)floor(ldexp(p, 32));
}

/* The paper's approximations of e^x (section 2.4, Figure 7, Appendix), as an
 * optional acceptance mode.  Both read a 32-bit integer i as the float with
 * the same bits, F(i) = (1 + frac(y)) 2^floor(y) for i = 2^23 (y + 127): a
 * linear interpolation of 2^y between integer y.
 *   fast:     e^x ~ 2 ln^2 2 F(round(2^23 x log2 e) + 127 * 2^23), the factor
 *             making the mean relative error zero; 0 below x = -126 ln 2.
 *   accurate: e^x ~ (2 ln^2 2 F(round(2^25 x log2 e) + 127 * 2^23))^(1/4)
 *             (F then interpolates 2^(4y), exact at four times the points);
 *             0 below x = -31.5 ln 2.
 * Readings: every step in FP32 (x rounded from FP64, products rounded to
 * nearest, the integer by round-half-even), and the fourth root taken
 * exactly (two correctly rounded square roots) where the paper uses an
 * approximate reciprocal square root, whose result is implementation
 * defined. */
static float orc_float_of_bits(uint32_t b)
{
    float f;
    memcpy(&f, &b, sizeof f);
    return f;
}

float orc_exp_approx(float x, int32_t accurate)
{
    const double ln2 = 0.69314718055994530942, log2e = 1.44269504088896340736;
    const float scale = (float)(2.0 * ln2 * ln2);
    if (!accurate) {
        if (x < (float)(-126.0 * ln2))
            return 0.0f;
        const float a = x * (float)(8388608.0 * log2e);
        const int32_t n = (int32_t)lrintf(a);
        return orc_float_of_bits((uint32_t)(n + 0x3F800000)) * scale;
    }
    if (x < (float)(-31.5 * ln2))
        return 0.0f;
    const float a = x * (float)(33554432.0 * log2e);
    const int32_t n = (int32_t)lrintf(a);
    const float g = orc_float_of_bits((uint32_t)(n + 0x3F800000)) * scale;
    return sqrtf(sqrtf(g));
}

/* Flip threshold of acceptance mode `mode` (0 exact, 1 fast, 2 accurate):
 * floor(2^32 min(1, e(-2 beta k))), e the mode's exponential; an estimate of
 * 1 or more becomes 2^32 - 1 (the table holds 32 bits). */
uint32_t orc_flip_threshold_mode(double beta, int64_t k, int32_t mode)
{
    if (mode == 0)
        return orc_flip_threshold(beta, k);
    const float p = orc_exp_approx((float)(-2.0 * beta * (double)k), mode == 2);
    const double t = floor(ldexp((double)p, 32));
    return t >= 4294967295.0 ? 0xFFFFFFFFu : (uint32_t)t;
}

/* S(d) = floor(2^32 exp(-dbeta d)) for d >= 1, dbeta = beta_{k+1} - beta_k. */
uint32_t orc_swap_threshold(double dbeta, int64_t d)
{
    double p = exp(-dbeta * (double)d);
    return (uint32_t)floor(ldexp(p, 32));
}

/* A deterministic exponential for the split-coupling PT rule below, whose
 * argument z = dbeta dE + dK dC is real-valued and too varied to tabulate on
 * the host: the same FP64 operations, in the same order and without fused
 * multiply-adds, give the same bits on any IEEE machine.
 *   Cody & Waite's reduction (Software Manual for the Elementary Functions,
 *   1980): x = n ln 2 + r with n = round-half-even(x / ln 2) and ln 2 split
 *   into a head of 32 significant bits (so n * head is exact) and a tail;
 *   |r| <= ln(2)/2 up to rounding.
 *   e^r by its Taylor series to degree 13 (truncation below r^14 / 14! <
 *   4e-18), Horner order, coefficients 1/k! rounded to nearest.
 *   e^x = e^r 2^n, exact while the result stays normal; x < -708 returns 0
 *   (every threshold built from it is 0 long before that).
 * Constants: head = ln 2 truncated to 32 significant bits, tail = ln 2 - head
 * rounded to FP64, 1/ln 2 rounded to FP64. */
double orc_exp_det(double x)
{
    static const double inv_ln2 = 0x1.71547652b82fep+0;
    static const double ln2_hi = 0x1.62e42fee00000p-1;
    static const double ln2_lo = 0x1.a39ef35793c76p-33;
    static const double inv_fact[14] = {
        0x1p+0, 0x1p+0, 0x1p-1, 0x1.5555555555555p-3, 0x1.5555555555555p-5,
        0x1.1111111111111p-7, 0x1.6c16c16c16c17p-10, 0x1.a01a01a01a01ap-13,
        0x1.a01a01a01a01ap-16, 0x1.71de3a556c734p-19, 0x1.27e4fb7789f5cp-22,
        0x1.ae64567f544e4p-26, 0x1.1eed8eff8d898p-29, 0x1.6124613a86d09p-33};
    if (x < -708.0)
        return 0.0;
    if (x > 709.0)
        return INFINITY;
    /* volatile keeps every product and sum rounded on its own (no contraction) */
    volatile double t = x * inv_ln2;
    const double n = nearbyint(t);
    volatile double a = n * ln2_hi;
    volatile double b = n * ln2_lo;
    volatile double r = (x - a) - b;
    volatile double p = inv_fact[13];
    for (int k = 12; k >= 0; k--) {
        volatile double pr = p * r;
        p = pr + inv_fact[k];
    }
    return ldexp(p, (int)n);
}

/* A 32-bit acceptance threshold: floor(2^32 p) for a probability p, held to
 * 2^32 - 1 when p rounds to 1 (or more). */
static uint32_t orc_threshold_of(double p)
{
    const double t = floor(ldexp(p, 32));
    return t >= 4294967295.0 ? 0xFFFFFFFFu : (uint32_t)t;
}

/* The exponents of the split-coupling rules, each product rounded on its own:
 * a flip of spin s has z = 2 (beta k_s + K k_tau), k_s = s f_space and
 * k_tau = s tau; a swap of the states at temperatures k, k+1 has
 * z = dbeta dE + dK dC, dE and dC the lower-temperature state's energy and
 * Trotter sum minus the upper one's. */
static double flip_z(double beta, double K, int64_t ks, int64_t kt)
{
    volatile double a = beta * (double)ks;
    volatile double b = K * (double)kt;
    return 2.0 * (a + b);
}

static double swap_z(double dbeta, double dK, int64_t dE, int64_t dC)
{
    volatile double a = dbeta * (double)dE;
    volatile double b = dK * (double)dC;
    return a + b;
}

/* Flip threshold with split couplings: floor(2^32 exp(-z)) with libm's exp
 * (the FP64 expression a host-built table uses), held to 2^32 - 1, and
 * 2^32 - 1 for z <= 0.  The flip is taken iff the threshold is 2^32 - 1 or
 * the word u is below it. */
uint32_t orc_trotter_flip_threshold(double beta, double K, int64_t ks, int64_t kt)
{
    const double z = flip_z(beta, K, ks, kt);
    return z <= 0.0 ? 0xFFFFFFFFu : orc_threshold_of(exp(-z));
}

/* Swap threshold with split couplings: floor(2^32 e^-z) with the
 * deterministic exponential, held to 2^32 - 1, and 2^32 - 1 for z <= 0; the
 * swap is taken iff the threshold is 2^32 - 1 or the word u is below it. */
uint32_t orc_trotter_swap_threshold(double dbeta, double dK, int64_t dE, int64_t dC)
{
    const double z = swap_z(dbeta, dK, dE, dC);
    return z <= 0.0 ? 0xFFFFFFFFu : orc_threshold_of(orc_exp_det(-z));
}

/* ----------------------------------------------------- energy and fields */
/* f_i = h_i + sum_j J_ij s_j (the quantity Figure 6 keeps up to date). */
void orc_fields(int32_t n, const int32_t* row_ptr, const int32_t* col,
                const int32_t* J, const int32_t* h, const int8_t* s, int64_t* f)
{
    for (int32_t i = 0; i < n; i++) {
        int64_t acc = h[i];
        for (int32_t e = row_ptr[i]; e < row_ptr[i + 1]; e++)
            acc += (int64_t)J[e] * (int64_t)s[col[e]];
        f[i] = acc;
    }
}

/* Cost function of section 1, each undirected edge once (CSR holds both
 * directions, so the pair term takes j > i only). */
int64_t orc_energy(int32_t n, const int32_t* row_ptr, const int32_t* col,
                   const int32_t* J, const int32_t* h, const int8_t* s)
{
    int64_t e = 0;
    for (int32_t i = 0; i < n; i++) {
        e -= (int64_t)h[i] * s[i];
        for (int32_t k = row_ptr[i]; k < row_ptr[i + 1]; k++)
            if (col[k] > i)
                e -= (int64_t)J[k] * s[i] * s[col[k]];
    }
    return e;
}

/* ------------------------------------------------------------- simulation */
typedef struct {
    /* graph */
    int32_t n, slice;
    int32_t *row_ptr, *col, *J, *h;
    int64_t kmax; /* largest possible |f_i| */
    /* ladder */
    int32_t R;
    double* beta;          /* [R] ascending */
    uint32_t** thr;        /* [R][kmax+1], thr[k][0] unused */
    /* rng */
    uint32_t seed, inst;
    int32_t mode;          /* 0 = MT19937, 1 = Philox4x32-10 */
    orc_mt* mt;            /* [R] replica streams (mode 0) */
    orc_mt swap_mt;        /* swap stream (mode 0) */
    /* state */
    int8_t* s;             /* [R][n] */
    int64_t* f;            /* [R][n] */
    int64_t* E;            /* [R] */
    int32_t* temp_of_slot; /* [R] */
    int32_t* slot_of_temp; /* [R] */
    uint64_t* swap_acc;    /* [R-1] */
    uint64_t sweeps, passes;
    int32_t threads;
    /* split couplings (orc_sim_set_trotter): 0 = off */
    int32_t split;
    double* K;             /* [R] Trotter coupling per temperature index */
    int64_t* C;            /* [R] -sum over Trotter pairs of s s' */
} orc_sim;

/* ------------------------------------------- split space / Trotter parts */
/* With split couplings an edge (i, j) is a Trotter edge when i and j lie in
 * different slices (i / S != j / S) and a spatial edge otherwise.  The
 * spatial part keeps the graph's J; the Trotter part counts every pair with
 * unit weight and the per-temperature coupling K_k instead of J. */
static int same_slice(const orc_sim* m, int32_t i, int32_t j)
{
    return i / m->slice == j / m->slice;
}

/* f_i = h_i + sum over spatial neighbours of J_ij s_j. */
static void split_fields(const orc_sim* m, const int8_t* s, int64_t* f)
{
    for (int32_t i = 0; i < m->n; i++) {
        int64_t acc = m->h[i];
        for (int32_t e = m->row_ptr[i]; e < m->row_ptr[i + 1]; e++)
            if (same_slice(m, i, m->col[e]))
                acc += (int64_t)m->J[e] * (int64_t)s[m->col[e]];
        f[i] = acc;
    }
}

/* E_space = -sum_i h_i s_i - sum over spatial pairs J s s' (each pair once). */
static int64_t split_energy(const orc_sim* m, const int8_t* s)
{
    int64_t e = 0;
    for (int32_t i = 0; i < m->n; i++) {
        e -= (int64_t)m->h[i] * s[i];
        for (int32_t k = m->row_ptr[i]; k < m->row_ptr[i + 1]; k++)
            if (m->col[k] > i && same_slice(m, i, m->col[k]))
                e -= (int64_t)m->J[k] * s[i] * s[m->col[k]];
    }
    return e;
}

/* C = -sum over Trotter pairs of s s' (each pair once). */
static int64_t split_trotter_sum(const orc_sim* m, const int8_t* s)
{
    int64_t c = 0;
    for (int32_t i = 0; i < m->n; i++)
        for (int32_t k = m->row_ptr[i]; k < m->row_ptr[i + 1]; k++)
            if (m->col[k] > i && !same_slice(m, i, m->col[k]))
                c -= (int64_t)s[i] * s[m->col[k]];
    return c;
}

/* tau_i = sum over Trotter neighbours of s_j. */
static int64_t split_tau(const orc_sim* m, const int8_t* s, int32_t i)
{
    int64_t t = 0;
    for (int32_t e = m->row_ptr[i]; e < m->row_ptr[i + 1]; e++)
        if (!same_slice(m, i, m->col[e]))
            t += s[m->col[e]];
    return t;
}

/* Fields, energy (and Trotter sum) of slot r from its spins. */
static void refresh_replica(orc_sim* m, int32_t r)
{
    const int8_t* s = m->s + (int64_t)r * m->n;
    int64_t* f = m->f + (int64_t)r * m->n;
    if (m->split) {
        split_fields(m, s, f);
        m->E[r] = split_energy(m, s);
        m->C[r] = split_trotter_sum(m, s);
    } else {
        orc_fields(m->n, m->row_ptr, m->col, m->J, m->h, s, f);
        m->E[r] = orc_energy(m->n, m->row_ptr, m->col, m->J, m->h, s);
    }
}

static uint32_t init_word(orc_sim* m, int32_t r, int32_t i)
{
    if (m->mode == 0)
        return orc_mt_next(&m->mt[r]);
    int32_t t = i / m->slice, q = i % m->slice;
    return philox_word(m->seed, (uint32_t)r, (uint32_t)((t >> 2) * m->slice + q), 0u,
                       m->inst, 3u, t & 3);
}

/* Figure 1 on one replica, with the Figure 6 neighbour update, repeated for
 * `nsweeps` sweeps.  Philox words depend on the instance sweep counter, so
 * the block starts from counter `c0` (replicas of one block run
 * concurrently, each with its own copy of the counter). */
static void sweep_replica_block(orc_sim* m, int32_t r, uint64_t c0, int64_t nsweeps)
{
    int8_t* s = m->s + (int64_t)r * m->n;
    int64_t* f = m->f + (int64_t)r * m->n;
    const uint32_t* T = m->thr[m->temp_of_slot[r]];
    const double beta = m->beta[m->temp_of_slot[r]];
    const double K = m->split ? m->K[m->temp_of_slot[r]] : 0.0;
    for (int64_t c = 0; c < nsweeps; c++) {
        int64_t dE = 0, dC = 0;
        uint32_t sweep_id = (uint32_t)(c0 + (uint64_t)c);
        for (int32_t i = 0; i < m->n; i++) {
            uint32_t u;
            if (m->mode == 0) {
                u = orc_mt_next(&m->mt[r]);
            } else {
                int32_t t = i / m->slice, q = i % m->slice;
                u = philox_word(m->seed, (uint32_t)r, (uint32_t)((t >> 2) * m->slice + q),
                                sweep_id, m->inst, 0u, t & 3);
            }
            int64_t k = (int64_t)s[i] * f[i];
            int64_t kt = 0;
            int accept;
            if (m->split) {
                /* split couplings: z = 2 s (beta f_space + K tau) */
                kt = (int64_t)s[i] * split_tau(m, s, i);
                const uint32_t thr = orc_trotter_flip_threshold(beta, K, k, kt);
                accept = (thr == 0xFFFFFFFFu) || (u < thr);
            } else {
                accept = (k <= 0) || (u < T[k]);
            }
            if (accept) {
                int64_t two_s = 2 * (int64_t)s[i];
                for (int32_t e = m->row_ptr[i]; e < m->row_ptr[i + 1]; e++)
                    if (!m->split || same_slice(m, i, m->col[e]))
                        f[m->col[e]] -= two_s * m->J[e];
                s[i] = (int8_t)(-s[i]);
                dE += 2 * k;
                dC += 2 * kt;
            }
        }
        m->E[r] += dE;
        if (m->split)
            m->C[r] += dC;
    }
}

typedef struct {
    orc_sim* m;
    int32_t r0, r1;
    uint64_t c0;
    int64_t nsweeps;
} block_job;

static void* block_worker(void* arg)
{
    block_job* jb = (block_job*)arg;
    for (int32_t r = jb->r0; r < jb->r1; r++)
        sweep_replica_block(jb->m, r, jb->c0, jb->nsweeps);
    return NULL;
}

/* n sweeps of every replica with no PT pass in between (replicas are
 * independent, so they run on the thread pool). */
void orc_sim_sweep(orc_sim* m, int64_t nsweeps)
{
    if (nsweeps <= 0)
        return;
    int32_t nt = m->threads < m->R ? m->threads : m->R;
    if (nt <= 1) {
        for (int32_t r = 0; r < m->R; r++)
            sweep_replica_block(m, r, m->sweeps, nsweeps);
    } else {
        pthread_t* th = (pthread_t*)malloc(sizeof(pthread_t) * nt);
        block_job* jobs = (block_job*)malloc(sizeof(block_job) * nt);
        for (int32_t w = 0; w < nt; w++) {
            jobs[w].m = m;
            jobs[w].r0 = (int32_t)((int64_t)m->R * w / nt);
            jobs[w].r1 = (int32_t)((int64_t)m->R * (w + 1) / nt);
            jobs[w].c0 = m->sweeps;
            jobs[w].nsweeps = nsweeps;
            pthread_create(&th[w], NULL, block_worker, &jobs[w]);
        }
        for (int32_t w = 0; w < nt; w++)
            pthread_join(th[w], NULL);
        free(th);
        free(jobs);
    }
    m->sweeps += (uint64_t)nsweeps;
}

/* One PT pass (parity = pass count mod 2). */
void orc_sim_pt(orc_sim* m)
{
    uint32_t p = (uint32_t)m->passes;
    for (int32_t k = (int32_t)(m->passes & 1u); k + 1 < m->R; k += 2) {
        uint32_t u;
        if (m->mode == 0) {
            u = orc_mt_next(&m->swap_mt);
        } else {
            uint32_t j = (uint32_t)(k >> 1);
            u = philox_word(m->seed, 0xFFFFFFFFu, j >> 2, p, m->inst, 1u, (int)(j & 3u));
        }
        int32_t a = m->slot_of_temp[k], b = m->slot_of_temp[k + 1];
        int64_t d = m->E[a] - m->E[b];
        int accept;
        if (m->split) {
            const uint32_t thr = orc_trotter_swap_threshold(m->beta[k + 1] - m->beta[k],
                                                            m->K[k + 1] - m->K[k], d, m->C[a] - m->C[b]);
            accept = (thr == 0xFFFFFFFFu) || (u < thr);
        } else {
            accept = (d <= 0) || (u < orc_swap_threshold(m->beta[k + 1] - m->beta[k], d));
        }
        if (accept) {
            m->slot_of_temp[k] = b;
            m->slot_of_temp[k + 1] = a;
            m->temp_of_slot[a] = k + 1;
            m->temp_of_slot[b] = k;
            m->swap_acc[k]++;
        }
    }
    m->passes++;
}

/* n sweeps; after every `swap_every`-th sweep of this call, one PT pass
 * (swap_every <= 0: no PT). */
void orc_sim_run(orc_sim* m, int64_t nsweeps, int32_t swap_every)
{
    if (swap_every <= 0) {
        orc_sim_sweep(m, nsweeps);
        return;
    }
    int64_t done = 0;
    while (done < nsweeps) {
        int64_t chunk = swap_every;
        if (chunk > nsweeps - done)
            chunk = nsweeps - done;
        orc_sim_sweep(m, chunk);
        done += chunk;
        if (chunk == swap_every)
            orc_sim_pt(m);
    }
}

orc_sim* orc_sim_create(int32_t n, const int32_t* row_ptr, const int32_t* col,
                        const int32_t* J, const int32_t* h, int32_t slice, int32_t R,
                        const double* beta, uint32_t seed, uint32_t inst, int32_t mode,
                        int32_t threads)
{
    orc_sim* m = (orc_sim*)calloc(1, sizeof(orc_sim));
    int32_t nnz = row_ptr[n];
    m->n = n;
    m->slice = slice > 0 ? slice : n;
    m->row_ptr = (int32_t*)malloc(sizeof(int32_t) * (n + 1));
    m->col = (int32_t*)malloc(sizeof(int32_t) * (nnz > 0 ? nnz : 1));
    m->J = (int32_t*)malloc(sizeof(int32_t) * (nnz > 0 ? nnz : 1));
    m->h = (int32_t*)malloc(sizeof(int32_t) * (n > 0 ? n : 1));
    memcpy(m->row_ptr, row_ptr, sizeof(int32_t) * (n + 1));
    if (nnz > 0) {
        memcpy(m->col, col, sizeof(int32_t) * nnz);
        memcpy(m->J, J, sizeof(int32_t) * nnz);
    }
    if (n > 0)
        memcpy(m->h, h, sizeof(int32_t) * n);
    m->kmax = 0;
    for (int32_t i = 0; i < n; i++) {
        int64_t b = llabs((long long)h[i]);
        for (int32_t e = row_ptr[i]; e < row_ptr[i + 1]; e++)
            b += llabs((long long)J[e]);
        if (b > m->kmax)
            m->kmax = b;
    }
    m->R = R;
    m->beta = (double*)malloc(sizeof(double) * R);
    memcpy(m->beta, beta, sizeof(double) * R);
    m->thr = (uint32_t**)malloc(sizeof(uint32_t*) * R);
    for (int32_t k = 0; k < R; k++) {
        m->thr[k] = (uint32_t*)malloc(sizeof(uint32_t) * (size_t)(m->kmax + 1));
        m->thr[k][0] = 0; /* never read: k <= 0 flips unconditionally */
        for (int64_t x = 1; x <= m->kmax; x++)
            m->thr[k][x] = orc_flip_threshold(beta[k], x);
    }
    m->seed = seed;
    m->inst = inst;
    m->mode = mode;
    m->s = (int8_t*)malloc((size_t)R * (n > 0 ? n : 1));
    m->f = (int64_t*)malloc(sizeof(int64_t) * (size_t)R * (n > 0 ? n : 1));
    m->E = (int64_t*)malloc(sizeof(int64_t) * R);
    m->temp_of_slot = (int32_t*)malloc(sizeof(int32_t) * R);
    m->slot_of_temp = (int32_t*)malloc(sizeof(int32_t) * R);
    m->swap_acc = (uint64_t*)calloc(R > 1 ? R - 1 : 1, sizeof(uint64_t));
    if (mode == 0) {
        m->mt = (orc_mt*)malloc(sizeof(orc_mt) * R);
        for (int32_t r = 0; r < R; r++)
            orc_mt_seed(&m->mt[r], seed + (uint32_t)r);
        orc_mt_seed(&m->swap_mt, seed + (uint32_t)R);
    }
    for (int32_t r = 0; r < R; r++) {
        int8_t* s = m->s + (int64_t)r * n;
        for (int32_t i = 0; i < n; i++)
            s[i] = (init_word(m, r, i) >> 31) ? (int8_t)1 : (int8_t)-1;
        refresh_replica(m, r);
        m->temp_of_slot[r] = r;
        m->slot_of_temp[r] = r;
    }
    if (threads <= 0) {
        long c = sysconf(_SC_NPROCESSORS_ONLN);
        threads = c > 0 ? (int32_t)c : 1;
    }
    m->threads = threads;
    return m;
}

void orc_sim_read(const orc_sim* m, int8_t* spins, int64_t* fields, int64_t* energy,
                  int32_t* temp_of_slot, uint64_t* counters, uint64_t* swap_acc)
{
    size_t rn = (size_t)m->R * (size_t)m->n;
    if (spins)
        memcpy(spins, m->s, rn);
    if (fields)
        memcpy(fields, m->f, rn * sizeof(int64_t));
    if (energy)
        memcpy(energy, m->E, sizeof(int64_t) * m->R);
    if (temp_of_slot)
        memcpy(temp_of_slot, m->temp_of_slot, sizeof(int32_t) * m->R);
    if (counters) {
        counters[0] = m->sweeps;
        counters[1] = m->passes;
    }
    if (swap_acc && m->R > 1)
        memcpy(swap_acc, m->swap_acc, sizeof(uint64_t) * (m->R - 1));
}

int32_t orc_sim_threads(const orc_sim* m) { return m->threads; }

/* Rebuild the flip thresholds of every temperature in acceptance mode `mode`
 * (0 exact, 1 fast, 2 accurate exponential of section 2.4). */
void orc_sim_set_acceptance(orc_sim* m, int32_t mode)
{
    for (int32_t k = 0; k < m->R; k++)
        for (int64_t x = 1; x <= m->kmax; x++)
            m->thr[k][x] = orc_flip_threshold_mode(m->beta[k], x, mode);
}

void orc_sim_destroy(orc_sim* m)
{
    if (!m)
        return;
    for (int32_t k = 0; k < m->R; k++)
        free(m->thr[k]);
    free(m->thr);
    free(m->beta);
    free(m->row_ptr);
    free(m->col);
    free(m->J);
    free(m->h);
    free(m->s);
    free(m->f);
    free(m->E);
    free(m->temp_of_slot);
    free(m->slot_of_temp);
    free(m->swap_acc);
    free(m->mt);
    free(m->K);
    free(m->C);
    free(m);
}

/* Overwrite the spins of slot r (tests start chains from chosen states);
 * fields and energy are recomputed from scratch. */
void orc_sim_set_spins(orc_sim* m, int32_t r, const int8_t* spins)
{
    int8_t* s = m->s + (int64_t)r * m->n;
    memcpy(s, spins, (size_t)m->n);
    refresh_replica(m, r);
}

/* Switch to split couplings (space and Trotter parts weighted apart): the
 * state at temperature index k then follows exp(-beta_k E_space - K_k C),
 * C = -sum over Trotter pairs of s s'.  Fields become spatial only and the
 * energy the spatial energy; both are rebuilt from the current spins.  The
 * flip rule uses libm's exp (as a host-built table would), the swap rule the
 * deterministic orc_exp_det.  K holds R values, by temperature index. */
void orc_sim_set_trotter(orc_sim* m, const double* K)
{
    if (!m->K)
        m->K = (double*)malloc(sizeof(double) * m->R);
    if (!m->C)
        m->C = (int64_t*)calloc(m->R, sizeof(int64_t));
    memcpy(m->K, K, sizeof(double) * m->R);
    m->split = 1;
    for (int32_t r = 0; r < m->R; r++)
        refresh_replica(m, r);
}

/* Trotter sums C of every slot (split couplings only; zeros otherwise). */
void orc_sim_read_trotter(const orc_sim* m, int64_t* C)
{
    for (int32_t r = 0; r < m->R; r++)
        C[r] = m->split ? m->C[r] : 0;
}
