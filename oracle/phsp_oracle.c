/*
 * phsp_oracle.c -- CPU ORACLE for the phase-space Monte Carlo.  TEST INFRASTRUCTURE ONLY.
 *
 * A plain, slow, single-threaded implementation of what the CUDA path computes, written
 * to be checked by eye against the method.  Only the test suite, the smoke check and the
 * benchmark's CPU-baseline / reference arm load it; the product library never does, and
 * this file shares no code, header, table or constant generator with the CUDA sources.
 *
 * Method: Hydra, section 4.2 "Phase-Space Monte Carlo" -- the Raubold-Lynch method of
 * F. James, "Monte Carlo Phase Space", CERN 68-15 (1968): a parent of mass M at rest
 * decays to n daughters through a chain of n-1 two-body decays; the n-2 intermediate
 * invariant masses come from sorted uniform numbers, each two-body decay is isotropic in
 * its own rest frame, and each event carries a weight proportional to the product of the
 * two-body momenta ("weighted samples", section 4.2).  4-vectors are (E, px, py, pz),
 * energy first, as in Listing 4's Vector4R(mother_mass, 0, 0, 0); events are stored as a
 * structure of arrays, one array per daughter component (section 2 and section 3.4).
 *
 * Readings of points the paper leaves open (each one is listed with its reason in the
 * design notes of the repository):
 *   R1  random numbers: Philox4x32-10 (Salmon, Moraes, Dror, Shaw, SC'11).  Key =
 *       (seed low word, seed high word); draw d of event e is word d%4 of the block with
 *       counter (e low, e high, d/4, 0).  Draws 0..n-3 are the mass draws, then for each
 *       top-down step j = 0..n-2 a cos(theta) draw (n-2+2j) and a phi draw (n-1+2j).
 *   R2  a 32-bit draw x maps to u = (x + 1/2) 2^-32, inside (0,1) and exact in FP64.
 *   R3  construction order: top-down (the parent decays first), each two-body decay in the
 *       rest frame of its subsystem, taken to the lab by a pure boost.
 *   R4  weight: w = C_n * prod_k p_k, C_n = pi^(n-1) 2^(n-2) T^(n-2) / ((n-2)! M), so that
 *       E[w] is the Lorentz-invariant phase-space volume
 *       R_n = Int prod_i d^3p_i/(2E_i) delta^4(P - sum_i p_i)  (no 2 pi factors).
 *   R5  the two-body momentum uses Kallen's lambda written as the product of its four
 *       factors, the first of which is the kinetic gap Delta_k (no cancellation).
 *   R6  the Dalitz matrix element is |BW(s12; a) + c BW(s23; b)|^2 with the constant-width
 *       relativistic Breit-Wigner BW(s; m0, G) = 1/(m0^2 - s - i m0 G).
 *
 * The file is compiled twice: REAL = double (symbols oracle_*) and, with -DORACLE_LD,
 * REAL = long double (symbols oracle_ld_*), so tests can state the oracle's own rounding
 * error.  Build flags: -O2 -ffp-contract=off (no fused multiply-add, no reassociation).
 */
#include <stdint.h>
#include <stdlib.h>
#include <tgmath.h>

#ifdef ORACLE_LD
typedef long double real;
#define API(name) oracle_ld_##name
#define PI_R 3.141592653589793238462643383279502884L
#else
typedef double real;
#define API(name) oracle_##name
#define PI_R 3.141592653589793238462643383279502884
#endif

#define NMAX 10

/* ------------------------------------------------------------------------------------ */
/* R1: Philox4x32-10 from its published definition (SC'11, "Parallel random numbers: as  */
/* easy as 1, 2, 3").  One round: two 32x32->64 products of the multipliers with counter  */
/* words 0 and 2; the high halves are xored with the other counter words and the key.     */
/* The key is bumped by the Weyl constants between rounds.                                */
/* ------------------------------------------------------------------------------------ */
static const uint32_t PHILOX_M0 = 0xD2511F53u, PHILOX_M1 = 0xCD9E8D57u;
static const uint32_t PHILOX_W0 = 0x9E3779B9u, PHILOX_W1 = 0xBB67AE85u;

void API(philox4x32_10)(const uint32_t ctr_in[4], const uint32_t key_in[2], uint32_t out[4])
{
    uint32_t c[4] = {ctr_in[0], ctr_in[1], ctr_in[2], ctr_in[3]};
    uint32_t k[2] = {key_in[0], key_in[1]};
    for (int round = 0; round < 10; ++round) {
        if (round > 0) {
            k[0] += PHILOX_W0;
            k[1] += PHILOX_W1;
        }
        uint64_t prod0 = (uint64_t)PHILOX_M0 * (uint64_t)c[0];
        uint64_t prod1 = (uint64_t)PHILOX_M1 * (uint64_t)c[2];
        uint32_t hi0 = (uint32_t)(prod0 >> 32), lo0 = (uint32_t)prod0;
        uint32_t hi1 = (uint32_t)(prod1 >> 32), lo1 = (uint32_t)prod1;
        uint32_t n0 = hi1 ^ c[1] ^ k[0];
        uint32_t n1 = lo1;
        uint32_t n2 = hi0 ^ c[3] ^ k[1];
        uint32_t n3 = lo0;
        c[0] = n0; c[1] = n1; c[2] = n2; c[3] = n3;
    }
    for (int i = 0; i < 4; ++i) out[i] = c[i];
}

/* Draw d of event `event` under key `seed` (R1). */
uint32_t API(draw)(uint64_t seed, uint64_t event, int d)
{
    uint32_t ctr[4] = {(uint32_t)event, (uint32_t)(event >> 32), (uint32_t)(d / 4), 0u};
    uint32_t key[2] = {(uint32_t)seed, (uint32_t)(seed >> 32)};
    uint32_t out[4];
    API(philox4x32_10)(ctr, key, out);
    return out[d % 4];
}

/* R2: u = (x + 1/2) * 2^-32. */
static real uniform_of(uint32_t x) { return ((real)x + (real)0.5) * (real)(1.0 / 4294967296.0); }

/* ------------------------------------------------------------------------------------ */
/* Setup shared by all events of one decay.                                              */
/* ------------------------------------------------------------------------------------ */
struct decay {
    int n;
    real M;           /* parent mass (at rest) */
    real m[NMAX];     /* daughter masses m_1..m_n stored at m[0..n-1] */
    real mu[NMAX];    /* mu[k-1] = m_1 + ... + m_k */
    real T;           /* kinetic energy M - sum m */
    real C;           /* weight constant C_n (R4) */
};

/* R4: C_n = pi^(n-1) 2^(n-2) T^(n-2) / ((n-2)! M). */
static real weight_constant(int n, real M, real T)
{
    real c = (real)1;
    for (int i = 0; i < n - 1; ++i) c *= PI_R;
    for (int i = 0; i < n - 2; ++i) c *= (real)2 * T;
    for (int i = 2; i <= n - 2; ++i) c /= (real)i;
    return c / M;
}

/* Returns 0 on success, -1 on bad arguments, -2 below threshold. */
static int setup_decay(struct decay *D, double M, int n, const double *masses)
{
    if (n < 2 || n > NMAX || !(M > 0.0)) return -1;
    D->n = n;
    D->M = (real)M;
    real sum = 0;
    for (int i = 0; i < n; ++i) {
        if (!(masses[i] >= 0.0)) return -1;
        D->m[i] = (real)masses[i];
        sum += D->m[i];
        D->mu[i] = sum;
    }
    D->T = D->M - sum;
    if (!(D->T > 0)) return -2;
    D->C = weight_constant(n, D->M, D->T);
    return 0;
}

double API(volume_factor)(double M, int n, const double *masses)
{
    struct decay D;
    if (setup_decay(&D, M, n, masses) != 0) return -1.0;
    return (double)D.C;
}

/* Pure boost of the 4-vector v = (E, px, py, pz) from the rest frame of a system of mass mq
 * to the frame in which that system has 4-momentum q:
 *   E' = (q0 E + q.p) / mq,   p' = p + q ((q.p) / (mq (q0 + mq)) + E / mq).            */
static void boost(const real q[4], real mq, const real v[4], real out[4])
{
    real qp = q[1] * v[1] + q[2] * v[2] + q[3] * v[3];
    real f = qp / (mq * (q[0] + mq)) + v[0] / mq;
    out[0] = (q[0] * v[0] + qp) / mq;
    out[1] = v[1] + q[1] * f;
    out[2] = v[2] + q[2] * f;
    out[3] = v[3] + q[3] * f;
}

/* ------------------------------------------------------------------------------------ */
/* One event of the Raubold-Lynch generator from its 3n-4 uniform variables u[0..3n-5]    */
/* (u[0..n-3] the intermediate-mass uniforms, then cos(theta) and phi uniforms per step). */
/* Writes p[i][0..3] = (E, px, py, pz) of daughter i+1 and returns the weight.            */
/* ------------------------------------------------------------------------------------ */
static real event_from_uniforms(const struct decay *D, const real *u, real p[][4])
{
    const int n = D->n;

    /* Step 2: sort the n-2 mass uniforms into ascending order (insertion sort). */
    real y[NMAX];
    for (int j = 0; j < n - 2; ++j) {
        real v = u[j];
        int i = j;
        while (i > 0 && y[i - 1] > v) { y[i] = y[i - 1]; --i; }
        y[i] = v;
    }

    /* Step 3: sorted uniforms r_0 = 0 < r_1 <= ... <= r_{n-2} < r_{n-1} = 1, the
     * intermediate invariant masses M_k of the subsystem of daughters 1..k,
     *   M_1 = m_1,  M_k = (m_1 + ... + m_k) + r_{k-1} T,  M_n = M,
     * and the kinetic gaps Delta_k = M_{k+1} - M_k - m_{k+1} = T (r_k - r_{k-1}).
     * (Arrays are indexed by k: Mk[k], r[k], gap[k].) */
    real r[NMAX + 1], Mk[NMAX + 1], gap[NMAX + 1];
    r[0] = 0;
    for (int j = 1; j <= n - 2; ++j) r[j] = y[j - 1];
    r[n - 1] = 1;
    Mk[1] = D->m[0];
    for (int k = 2; k <= n - 1; ++k) Mk[k] = D->mu[k - 1] + r[k - 1] * D->T;
    Mk[n] = D->M;
    for (int k = 1; k <= n - 1; ++k) gap[k] = D->T * (r[k] - r[k - 1]);

    /* Step 4 (R5): two-body momentum of the decay M_{k+1} -> M_k + m_{k+1},
     *   p_k = sqrt(lambda(M_{k+1}^2, M_k^2, m_{k+1}^2)) / (2 M_{k+1}),
     *   lambda = (M_{k+1} - M_k - m)(M_{k+1} + M_k + m)(M_{k+1} - M_k + m)(M_{k+1} + M_k - m)
     *          = Delta (Delta + 2M_k + 2m)(Delta + 2m)(Delta + 2M_k). */
    real pk[NMAX + 1];
    for (int k = 1; k <= n - 1; ++k) {
        real g = gap[k], a = Mk[k], b = D->m[k];
        real lam = g * (g + (real)2 * a + (real)2 * b) * (g + (real)2 * b) * (g + (real)2 * a);
        pk[k] = sqrt(lam) / ((real)2 * Mk[k + 1]);
    }

    /* Step 5 (R4): the event weight. */
    real w = D->C;
    for (int k = 1; k <= n - 1; ++k) w *= pk[k];

    /* Steps 6-7 (R3): top-down two-body decays.  Q is the lab 4-momentum of subsystem
     * k+1 (daughters 1..k+1), starting from the parent at rest.  Step j = n-1-k uses the
     * isotropic direction cos(theta) = 2u - 1, phi = 2 pi u'. */
    real Q[4] = {D->M, 0, 0, 0};
    for (int k = n - 1; k >= 1; --k) {
        int j = n - 1 - k;
        real c = (real)2 * u[n - 2 + 2 * j] - (real)1;
        real s = sqrt(((real)1 - c) * ((real)1 + c));
        real phi = (real)2 * PI_R * u[n - 1 + 2 * j];
        real dir[3] = {s * cos(phi), s * sin(phi), c};
        real q = pk[k];
        /* In the rest frame of subsystem k+1: subsystem k along +dir, daughter k+1 along -dir. */
        real sub[4] = {sqrt(q * q + Mk[k] * Mk[k]), q * dir[0], q * dir[1], q * dir[2]};
        real dau[4] = {sqrt(q * q + D->m[k] * D->m[k]), -q * dir[0], -q * dir[1], -q * dir[2]};
        real sub_lab[4], dau_lab[4];
        boost(Q, Mk[k + 1], sub, sub_lab);
        boost(Q, Mk[k + 1], dau, dau_lab);
        for (int c4 = 0; c4 < 4; ++c4) {
            p[k][c4] = dau_lab[c4]; /* daughter k+1 is stored at index k */
            Q[c4] = sub_lab[c4];
        }
    }
    for (int c4 = 0; c4 < 4; ++c4) p[0][c4] = Q[c4]; /* daughter 1 = subsystem 1 */
    return w;
}

/* One event from its Philox draws (R1): u_d = (x_d + 1/2) 2^-32 (R2), then the map above. */
static real one_event(const struct decay *D, uint64_t seed, uint64_t event, real p[][4])
{
    real u[3 * NMAX];
    for (int d = 0; d < 3 * D->n - 4; ++d) u[d] = uniform_of(API(draw)(seed, event, d));
    return event_from_uniforms(D, u, p);
}

/* Generate events event_offset .. event_offset+nevents-1 into the structure of arrays
 * out[(i*4 + c) * nevents + e] (daughter i, component c in (E, px, py, pz)) and w[e].
 * Returns 0, -1 (bad arguments) or -2 (below threshold). */
int API(generate)(double M, int n, const double *masses, uint64_t nevents, uint64_t seed,
                  uint64_t event_offset, real *out, real *w)
{
    struct decay D;
    int rc = setup_decay(&D, M, n, masses);
    if (rc != 0) return rc;
    real p[NMAX][4];
    for (uint64_t e = 0; e < nevents; ++e) {
        real we = one_event(&D, seed, event_offset + e, p);
        for (int i = 0; i < n; ++i)
            for (int c = 0; c < 4; ++c) out[((uint64_t)i * 4 + (uint64_t)c) * nevents + e] = p[i][c];
        w[e] = we;
    }
    return 0;
}

/* ------------------------------------------------------------------------------------ */
/* Matrix elements for phase-space integration (section 3 "phase-space Monte Carlo       */
/* integration"; R6).  params = (m0a, Ga, m0b, Gb, |c|, arg c).                          */
/* ------------------------------------------------------------------------------------ */
static real invariant_mass2(const real a[4], const real b[4])
{
    real E = a[0] + b[0], x = a[1] + b[1], y = a[2] + b[2], z = a[3] + b[3];
    return E * E - (x * x + y * y + z * z);
}

/* |BW(s12; m0a, Ga) + c BW(s23; m0b, Gb)|^2 with BW(s) = (m0^2 - s + i m0 G) / ((m0^2 - s)^2 + (m0 G)^2). */
static real dalitz_2bw(real s12, real s23, const double *par)
{
    real m0a = par[0], Ga = par[1], m0b = par[2], Gb = par[3], cm = par[4], ca = par[5];
    real xa = m0a * m0a - s12, ya = m0a * Ga, da = xa * xa + ya * ya;
    real xb = m0b * m0b - s23, yb = m0b * Gb, db = xb * xb + yb * yb;
    real re_a = xa / da, im_a = ya / da;
    real re_b = xb / db, im_b = yb / db;
    real re_c = cm * cos(ca), im_c = cm * sin(ca);
    real re = re_a + (re_c * re_b - im_c * im_b);
    real im = im_a + (re_c * im_b + im_c * re_b);
    return re * re + im * im;
}

double API(me_dalitz_2bw)(double s12, double s23, const double *params)
{
    return (double)dalitz_2bw((real)s12, (real)s23, params);
}

/* Phase-space integral of f = w |ME|^2 over events event_offset .. +nevents-1.
 * sums[0..3] = (sum f, sum f^2, sum w, sum w^2), accumulated in long double.
 * me: 0 = flat (|ME|^2 = 1), 1 = Dalitz two-Breit-Wigner (needs n = 3, 6 params).
 * Returns 0, -1 (bad arguments) or -2 (below threshold). */
int API(integrate)(double M, int n, const double *masses, uint64_t nevents, uint64_t seed,
                   uint64_t event_offset, int me, const double *params, int nparams,
                   double sums[4])
{
    struct decay D;
    int rc = setup_decay(&D, M, n, masses);
    if (rc != 0) return rc;
    if (me == 1 && (n != 3 || nparams < 6)) return -1;
    if (me != 0 && me != 1) return -1;
    long double sf = 0, sf2 = 0, sw = 0, sw2 = 0;
    real p[NMAX][4];
    for (uint64_t e = 0; e < nevents; ++e) {
        real w = one_event(&D, seed, event_offset + e, p);
        real me2 = 1;
        if (me == 1) me2 = dalitz_2bw(invariant_mass2(p[0], p[1]), invariant_mass2(p[1], p[2]), params);
        real f = w * me2;
        sf += f; sf2 += (long double)f * f;
        sw += w; sw2 += (long double)w * w;
    }
    sums[0] = (double)sf; sums[1] = (double)sf2; sums[2] = (double)sw; sums[3] = (double)sw2;
    return 0;
}

/* ------------------------------------------------------------------------------------ */
/* Moving mother (Listing 4, Generate(Mother, ...)): each event is generated in the parent */
/* rest frame as above and every daughter is then taken to the frame in which the parent */
/* has momentum (px, py, pz) and energy sqrt(M^2 + p^2) by the pure boost of boost().     */
/* mothers: NULL -> one momentum mother_p[3] for all events; otherwise per-event momenta  */
/* stored as mothers[c * mld + e], c = x, y, z.                                           */
/* ------------------------------------------------------------------------------------ */
int API(generate_boosted)(double M, int n, const double *masses, uint64_t nevents, uint64_t seed,
                          uint64_t event_offset, const double *mother_p, const double *mothers,
                          uint64_t mld, real *out, real *w)
{
    struct decay D;
    int rc = setup_decay(&D, M, n, masses);
    if (rc != 0) return rc;
    real p[NMAX][4];
    for (uint64_t e = 0; e < nevents; ++e) {
        real we = one_event(&D, seed, event_offset + e, p);
        real P[4];
        for (int c = 0; c < 3; ++c) P[c + 1] = mothers ? (real)mothers[(uint64_t)c * mld + e] : (real)mother_p[c];
        P[0] = sqrt(D.M * D.M + P[1] * P[1] + P[2] * P[2] + P[3] * P[3]);
        for (int i = 0; i < n; ++i) {
            real lab[4];
            boost(P, D.M, p[i], lab);
            for (int c = 0; c < 4; ++c) out[((uint64_t)i * 4 + (uint64_t)c) * nevents + e] = lab[c];
        }
        w[e] = we;
    }
    return 0;
}

/* ------------------------------------------------------------------------------------ */
/* Unweighting by accept-reject (section 4.2, "unweighted samples"): event e is kept when */
/* u_e w_max < w_e, u_e = (x + 1/2) 2^-32 with x the event's draw 3n-4 (the first draw    */
/* after those of its kinematics).  accept[e] = 1 or 0.  The weights are the oracle's.     */
/* ------------------------------------------------------------------------------------ */
int API(unweight)(double M, int n, const double *masses, uint64_t nevents, uint64_t seed,
                  uint64_t event_offset, double w_max, unsigned char *accept)
{
    struct decay D;
    int rc = setup_decay(&D, M, n, masses);
    if (rc != 0) return rc;
    if (!(w_max > 0.0)) return -1;
    real p[NMAX][4];
    for (uint64_t e = 0; e < nevents; ++e) {
        real we = one_event(&D, seed, event_offset + e, p);
        real u = uniform_of(API(draw)(seed, event_offset + e, 3 * n - 4));
        accept[e] = (unsigned char)(u * (real)w_max < we);
    }
    return 0;
}

/* ------------------------------------------------------------------------------------ */
/* Model evaluation on stored events (section 4.2, "evaluation of model"; section 3,     */
/* "parallel function evaluation"): f_e = w_e |ME|^2(p_e) for events given as the         */
/* structure of arrays ev[(i*4 + c) * ld + e] and weights w[e].  values[e] = f_e (if not  */
/* NULL); sums[0..3] = (sum f, sum f^2, sum w, sum w^2) in long double.  me as integrate.  */
/* ------------------------------------------------------------------------------------ */
int API(evaluate)(int n, uint64_t nevents, const double *ev, uint64_t ld, const double *w, int me,
                  const double *params, int nparams, double *values, double sums[4])
{
    if (n < 2 || n > NMAX) return -1;
    if (me == 1 && (n != 3 || nparams < 6)) return -1;
    if (me != 0 && me != 1) return -1;
    long double sf = 0, sf2 = 0, sw = 0, sw2 = 0;
    for (uint64_t e = 0; e < nevents; ++e) {
        real p[NMAX][4];
        for (int i = 0; i < n; ++i)
            for (int c = 0; c < 4; ++c) p[i][c] = (real)ev[((uint64_t)i * 4 + (uint64_t)c) * ld + e];
        real me2 = 1;
        if (me == 1) me2 = dalitz_2bw(invariant_mass2(p[0], p[1]), invariant_mass2(p[1], p[2]), params);
        real we = (real)w[e];
        real f = we * me2;
        if (values) values[e] = (double)f;
        sf += f; sf2 += (long double)f * f;
        sw += we; sw2 += (long double)we * we;
    }
    sums[0] = (double)sf; sums[1] = (double)sf2; sums[2] = (double)sw; sums[3] = (double)sw2;
    return 0;
}

/* ------------------------------------------------------------------------------------ */
/* VEGAS over the phase-space variables (section 3 "self-adaptive importance sampling",   */
/* section 4.1; G. P. Lepage, J. Comput. Phys. 27 (1978) 192, with the iteration and      */
/* grid refinement structure of GSL's vegas in importance-sampling mode).                  */
/*                                                                                          */
/* The integrand is F(u) = w(u) |ME|^2(event(u)) on the unit cube of the D = 3n-4 uniform  */
/* variables of event_from_uniforms, so Int F du = Int |ME|^2 dR_n.  Each dimension has a  */
/* grid of K bins (edges g[d][0] = 0 < ... < g[d][K] = 1).  Iteration i draws `calls`     */
/* points: y_d = (x + 1/2) 2^-32 from Philox draw d of sample s under counter (s low, s    */
/* high, d/4, i + 1) (stream i + 1; key = seed); bin b = floor(y K); u_d = g[b] + (y K - b) */
/* (g[b+1] - g[b]); Jacobian J = prod_d K (g[b+1] - g[b]); f = F(u) J.  The iteration's    */
/* estimate is the mean of f with variance (<f^2> - <f>^2)/(calls - 1); each bin collects  */
/* the sum of f^2 of its points.  Refinement per dimension: smooth the bin sums with       */
/* weights (1, 2, 1)/4 inside and (1, 1)/2 at the ends, turn each into the importance      */
/* weight ((r - 1)/ln r)^alpha with r = d_i / sum d (0 for an empty bin), and move the     */
/* edges so that every new bin holds an equal share of the total weight (linear within    */
/* the old bins).  Iterations from `skip` on are combined with weights 1/var: result =     */
/* sum(I_i/var_i)/sum(1/var_i), sigma = 1/sqrt(sum 1/var_i), chi2/dof over those          */
/* iterations.  K = 1 is plain Monte Carlo.                                                */
/* ------------------------------------------------------------------------------------ */
#define VEGAS_MAXD (3 * NMAX - 4)
#define VEGAS_MAXK 256

static void vegas_refine(double *g, const double *dsum, int K, double alpha)
{
    double d[VEGAS_MAXK], w[VEGAS_MAXK], tot = 0.0;
    if (K == 1) return;
    d[0] = (dsum[0] + dsum[1]) / 2.0;
    for (int i = 1; i < K - 1; ++i) d[i] = (dsum[i - 1] + 2.0 * dsum[i] + dsum[i + 1]) / 4.0;
    d[K - 1] = (dsum[K - 2] + dsum[K - 1]) / 2.0;
    for (int i = 0; i < K; ++i) tot += d[i];
    if (!(tot > 0.0)) return;
    double wtot = 0.0;
    for (int i = 0; i < K; ++i) {
        double r = d[i] / tot;
        w[i] = (r > 0.0 && r < 1.0) ? pow((r - 1.0) / log(r), alpha) : (r >= 1.0 ? 1.0 : 0.0);
        wtot += w[i];
    }
    if (!(wtot > 0.0)) return;
    double per = wtot / K, acc = 0.0, newg[VEGAS_MAXK + 1];
    int j = 0; /* old bin being consumed */
    newg[0] = 0.0;
    for (int i = 1; i < K; ++i) {
        double need = per * i;
        while (j < K - 1 && acc + w[j] < need) { acc += w[j]; ++j; }
        double frac = w[j] > 0.0 ? (need - acc) / w[j] : 0.0;
        if (frac > 1.0) frac = 1.0;
        if (frac < 0.0) frac = 0.0;
        newg[i] = g[j] + frac * (g[j + 1] - g[j]);
    }
    newg[K] = 1.0;
    for (int i = 0; i <= K; ++i) g[i] = newg[i];
}

int API(vegas)(double M, int n, const double *masses, uint64_t seed, int me, const double *params,
               int nparams, uint64_t calls, int iterations, int bins, double alpha, int skip,
               double *est, double *var, double *result, double *grid_out)
{
    struct decay D;
    int rc = setup_decay(&D, M, n, masses);
    if (rc != 0) return rc;
    if (me == 1 && (n != 3 || nparams < 6)) return -1;
    if ((me != 0 && me != 1) || bins < 1 || bins > VEGAS_MAXK || iterations < 1 || calls < 2) return -1;
    const int Dm = 3 * n - 4, K = bins;
    static double g[VEGAS_MAXD][VEGAS_MAXK + 1], dsum[VEGAS_MAXD][VEGAS_MAXK];
    for (int d = 0; d < Dm; ++d)
        for (int b = 0; b <= K; ++b) g[d][b] = (double)b / K;
    uint32_t key[2] = {(uint32_t)seed, (uint32_t)(seed >> 32)};
    double sw = 0.0, swi = 0.0, swi2 = 0.0;
    for (int it = 0; it < iterations; ++it) {
        for (int d = 0; d < Dm; ++d)
            for (int b = 0; b < K; ++b) dsum[d][b] = 0.0;
        long double sf = 0, sf2 = 0;
        for (uint64_t s = 0; s < calls; ++s) {
            real u[3 * NMAX], p[NMAX][4];
            int bin[3 * NMAX];
            double jac = 1.0;
            for (int d = 0; d < Dm; ++d) {
                uint32_t ctr[4] = {(uint32_t)s, (uint32_t)(s >> 32), (uint32_t)(d / 4), (uint32_t)(it + 1)};
                uint32_t out[4];
                API(philox4x32_10)(ctr, key, out);
                double y = ((double)out[d % 4] + 0.5) * (1.0 / 4294967296.0);
                int b = (int)(y * K);
                if (b >= K) b = K - 1;
                double width = g[d][b + 1] - g[d][b];
                u[d] = (real)(g[d][b] + (y * K - b) * width);
                jac *= K * width;
                bin[d] = b;
            }
            real w = event_from_uniforms(&D, u, p);
            real me2 = 1;
            if (me == 1) me2 = dalitz_2bw(invariant_mass2(p[0], p[1]), invariant_mass2(p[1], p[2]), params);
            double f = (double)(w * me2) * jac;
            sf += f;
            sf2 += (long double)f * f;
            for (int d = 0; d < Dm; ++d) dsum[d][bin[d]] += f * f;
        }
        double mean = (double)(sf / calls);
        double v = (double)((sf2 / calls - (long double)mean * mean) / (calls - 1));
        est[it] = mean;
        var[it] = v;
        if (it >= skip && v > 0.0) {
            sw += 1.0 / v;
            swi += mean / v;
            swi2 += mean * mean / v;
        }
        if (it < iterations - 1)
            for (int d = 0; d < Dm; ++d) vegas_refine(g[d], dsum[d], K, alpha);
    }
    double res = sw > 0.0 ? swi / sw : est[iterations - 1];
    int used = iterations - skip;
    result[0] = res;
    result[1] = sw > 0.0 ? 1.0 / sqrt(sw) : sqrt(var[iterations - 1]);
    result[2] = used > 1 ? (swi2 - res * res * sw) / (used - 1) : 0.0;
    if (grid_out)
        for (int d = 0; d < Dm; ++d)
            for (int b = 0; b <= K; ++b) grid_out[d * (K + 1) + b] = g[d][b];
    return 0;
}
