/*
 * qtb_oracle.c -- plain, slow FP64 CPU oracle of the QTB / QTB-PIMD hot path.
 *
 * TEST INFRASTRUCTURE.  Only the test-suite, the smoke check and the CPU
 * baseline leg of the benchmark may load this library.  It shares no code,
 * header, table or constant with the CUDA path; every quantity is written out
 * here from its definition.
 *
 * Method (Dammak, Hayoun, Brieuc, Geneste, "Nuclear quantum effects in
 * molecular dynamics simulations"):
 *   Eq. 3   ring-polymer effective potential: V/P per replica plus cyclic
 *           springs 1/2 m w_P^2 (r_s - r_{s+1})^2, w_P = sqrt(P)/(beta hbar)
 *   Eq. 4   bead equation of motion: -(1/P) grad V - spring force
 *   Eq. 5   primitive total-energy estimator
 *   Eqs. 6-8  Langevin equation with a coloured random force whose power
 *           spectral density is 2 m gamma theta(w,T)  (kappa_P for QTB-PIMD,
 *           Eq. 12, applied to the ring-polymer normal modes, Sec. 2.3)
 *   Eq. 11  normal-mode frequencies of the free ring polymer
 *   (Sec. 2.3) centroid-virial kinetic estimators of the ring polymer, which
 *           the paper does not print (it gives the primitive one, Eq. 5)
 *
 * Readings where the paper is silent (each also listed in the design notes):
 *   - the coloured noise is a zero-phase time-domain filter of white noise,
 *     eta_n = sum_{k=-K..K} h_|k| xi_{n-k}; the taps h come from the spectrum
 *     (computed by the numpy half of the oracle);
 *   - the white noise xi is Philox4x32-10 (Salmon et al., SC'11) + Box-Muller,
 *     counter = (lo32(n>>2), dof, 0, hi32(n>>2)), key = (lo32(seed),
 *     hi32(seed) ^ sys); the four 32-bit words give the normals of steps
 *     4q..4q+3: (w0,w1) -> cos/sin pair for 4q, 4q+1, (w2,w3) -> 4q+2, 4q+3;
 *   - the integrator is BAOAB: B(dt/2) in bead space, then A(dt/2) O(dt)
 *     A(dt/2) in normal-mode space (exact free ring-polymer rotation), force,
 *     B(dt/2);  O: v <- c1 v + sqrt((1-c1^2)/m) eta, c1 = exp(-gamma dt);
 *   - pair potential: energy-shifted Buckingham + damped shifted force
 *     Coulomb (Fennell & Gezelter 2006), all periodic images within r_c;
 *   - isothermal-isobaric runs (Sec. 2.1: the paper uses Quigley and Probert's
 *     Langevin extension to constant pressure, refs [11, 12], and prints no
 *     equations): isotropic Martyna-Tobias-Klein equations with Langevin
 *     friction and noise on the particles and on the cell,
 *       dr/dt = v + v_e r,   m dv/dt = F - alpha m v_e v - gamma m v + R,
 *       dV/dt = 3 V v_e,     dp_e/dt = G - gamma_e p_e + R_e,  v_e = p_e / W,
 *       G = 2 alpha K + Wvir - 3 V P_ext,  alpha = 1 + 3/N_f,  N_f = 3N,
 *     Wvir = sum over pairs of r_ij . F_ij; split as B_e(dt/2) B(dt/2) A(dt/2)
 *     O(dt) A(dt/2) force B(dt/2) B_e(dt/2), each B and A the exact solution of
 *     its linear equation; the cell's random force is Philox stream 1, dof 0.
 *     Stationary law: P(V) ~ V^N exp(-(U + P_ext V)/k_B T).
 *     Ring polymers (P > 1): the cell acts on each atom's centroid mode only
 *     (the internal modes, physical bead offsets from the centroid, do not
 *     scale with it), so the equations above hold for the centroid modes
 *     Q_0 = sqrt(P) rbar with K -> K_0, the centroid modes' kinetic energy, and
 *     Wvir -> W_cv = sum_i rbar_i . F_i = (1/P) sum_s Wvir_s - sum_i sum_s
 *     (r_i,s - rbar_i) . f_i,s (f = -(1/P) grad V, Eq. 4), the virial of a
 *     scaling of the centroids at fixed offsets; N_f = 3N.  B and the O of the
 *     modes as in the constant-volume step, the centroid's B and A with the
 *     cell's friction and drift factors.  Stationary law: the ring polymer's
 *     isothermal-isobaric distribution (for an ideal gas again V^N
 *     exp(-P_ext V / k_B T)).
 *
 * Units: A, fs, eV, u, e, K.
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

#define ORA_HBAR 0.6582119569           /* eV fs            (CODATA 2018) */
#define ORA_KB 8.617333262e-5           /* eV / K           (CODATA 2018) */
#define ORA_MVV2E 103.64269652680505    /* eV per u A^2 fs^-2              */
#define ORA_KE 14.3996454784            /* e^2/(4 pi eps0) in eV A         */
#define ORA_PI 3.14159265358979323846

#define ORA_NREC 23

/* ------------------------------------------------------------------------ */
/* Philox4x32-10, from its published definition: 10 rounds of
 *   (c0,c1,c2,c3) -> (hi(M1 c2) ^ c1 ^ k0, lo(M1 c2), hi(M0 c0) ^ c3 ^ k1, lo(M0 c0))
 * with the key bumped by the Weyl constants between rounds.                  */
void ora_philox4x32_10(const uint32_t ctr[4], const uint32_t key[2], uint32_t out[4])
{
    const uint32_t M0 = 0xD2511F53u, M1 = 0xCD9E8D57u;
    const uint32_t W0 = 0x9E3779B9u, W1 = 0xBB67AE85u;
    uint32_t c0 = ctr[0], c1 = ctr[1], c2 = ctr[2], c3 = ctr[3];
    uint32_t k0 = key[0], k1 = key[1];
    for (int r = 0; r < 10; ++r) {
        if (r > 0) { k0 += W0; k1 += W1; }
        uint64_t p0 = (uint64_t)M0 * (uint64_t)c0;
        uint64_t p1 = (uint64_t)M1 * (uint64_t)c2;
        uint32_t n0 = (uint32_t)(p1 >> 32) ^ c1 ^ k0;
        uint32_t n1 = (uint32_t)p1;
        uint32_t n2 = (uint32_t)(p0 >> 32) ^ c3 ^ k1;
        uint32_t n3 = (uint32_t)p0;
        c0 = n0; c1 = n1; c2 = n2; c3 = n3;
    }
    out[0] = c0; out[1] = c1; out[2] = c2; out[3] = c3;
}

/* floor(n / 4) for signed n */
static int64_t quad_of(int64_t n) { return (n >= 0) ? n / 4 : -((-n + 3) / 4); }

/* The four unit normals of steps 4q .. 4q+3 for one degree of freedom. */
static void white_quad(uint64_t seed, uint32_t sys, uint32_t dof, uint32_t stream,
                       int64_t q, double xi[4])
{
    uint64_t uq = (uint64_t)q;
    uint32_t ctr[4] = {(uint32_t)uq, dof, stream, (uint32_t)(uq >> 32)};
    uint32_t key[2] = {(uint32_t)seed, (uint32_t)(seed >> 32) ^ sys};
    uint32_t w[4];
    ora_philox4x32_10(ctr, key, w);
    const double two32 = 4294967296.0;
    for (int pr = 0; pr < 2; ++pr) {
        double u1 = ((double)w[2 * pr] + 1.0) / two32;     /* (0, 1] */
        double u2 = (double)w[2 * pr + 1] / two32;         /* [0, 1) */
        double r = sqrt(-2.0 * log(u1));
        double a = 2.0 * ORA_PI * u2;
        xi[2 * pr] = r * cos(a);
        xi[2 * pr + 1] = r * sin(a);
    }
}

/* One unit normal xi(n, dof). */
double ora_white(uint64_t seed, uint32_t sys, uint32_t dof, uint32_t stream, int64_t n)
{
    double xi[4];
    int64_t q = quad_of(n);
    white_quad(seed, sys, dof, stream, q, xi);
    return xi[n - 4 * q];
}

/* White normals for steps n0 .. n0+nsteps-1 of dofs 0 .. ndof-1: out[dof][step]. */
void ora_white_block(uint64_t seed, uint32_t sys, uint32_t stream, int ndof, int64_t n0,
                     int nsteps, double *out)
{
    for (int d = 0; d < ndof; ++d)
        for (int j = 0; j < nsteps; ++j)
            out[(size_t)d * nsteps + j] = ora_white(seed, sys, (uint32_t)d, stream, n0 + j);
}

/* Coloured noise eta(n, dof) = sum_{k=-K..K} h_|k| xi(n-k, dof), for steps
 * n0 .. n0+nsteps-1 and dofs 0 .. ndof-1: out[dof][step].  Direct sum. */
void ora_colored_block(uint64_t seed, uint32_t sys, int ndof, int64_t n0, int nsteps,
                       int K, const double *h, double *out)
{
    int span = nsteps + 2 * K;
    double *xi = (double *)malloc(sizeof(double) * (size_t)span);
    for (int d = 0; d < ndof; ++d) {
        for (int t = 0; t < span; ++t)
            xi[t] = ora_white(seed, sys, (uint32_t)d, 0, n0 - K + t);
        for (int j = 0; j < nsteps; ++j) {
            double acc = 0.0;
            /* xi(n - k) with n = n0 + j sits at t = j + K - k */
            for (int k = -K; k <= K; ++k)
                acc += h[k < 0 ? -k : k] * xi[j + K - k];
            out[(size_t)d * nsteps + j] = acc;
        }
    }
    free(xi);
}

/* ------------------------------------------------------------------------ */
/* Normal modes of the cyclic ring polymer (Sec. 2.3; Eq. 11 with w -> 0):
 * real discrete-Fourier basis, C[s][k]; frequencies 2 w_P sin(k pi / P).     */
void ora_nm_matrix(int P, double *C)
{
    for (int s = 0; s < P; ++s)
        for (int k = 0; k < P; ++k) {
            double v;
            if (k == 0)
                v = 1.0 / sqrt((double)P);
            else if (2 * k < P)
                v = sqrt(2.0 / P) * cos(2.0 * ORA_PI * (double)((s * k) % P) / P);
            else if (2 * k == P)
                v = ((s % 2) ? -1.0 : 1.0) / sqrt((double)P);
            else
                v = sqrt(2.0 / P) * sin(2.0 * ORA_PI * (double)((s * k) % P) / P);
            C[s * P + k] = v;
        }
}

void ora_nm_freqs(int P, double T, double *wk)
{
    double wP = sqrt((double)P) * ORA_KB * T / ORA_HBAR;
    for (int k = 0; k < P; ++k) wk[k] = 2.0 * wP * sin(ORA_PI * k / P);
}

/* ------------------------------------------------------------------------ */
/* Pair potential (Buckingham, energy-shifted, + DSF Coulomb).                */
typedef struct {
    int ntypes;
    const double *charge, *bA, *brho, *bC;
    double alpha, rc;
} ora_pairpot;

/* radial energy and force magnitude (-dV/dr) of one pair at distance r < rc */
static void pair_eval(const ora_pairpot *pp, int ti, int tj, double r, double *e, double *fr)
{
    int t = ti * pp->ntypes + tj;
    double A = pp->bA[t], rho = pp->brho[t], Cc = pp->bC[t];
    double rc = pp->rc, al = pp->alpha;
    double en = 0.0, f = 0.0;
    if (A != 0.0 || Cc != 0.0) {
        double ex = (A != 0.0) ? A * exp(-r / rho) : 0.0;
        double exc = (A != 0.0) ? A * exp(-rc / rho) : 0.0;
        double r6 = r * r * r * r * r * r, rc6 = rc * rc * rc * rc * rc * rc;
        en += ex - Cc / r6 - (exc - Cc / rc6);
        f += ((A != 0.0) ? ex / rho : 0.0) - 6.0 * Cc / (r6 * r);
    }
    double qq = ORA_KE * pp->charge[ti] * pp->charge[tj];
    if (qq != 0.0) {
        double twoapi = 2.0 * al / sqrt(ORA_PI);
        double erc = erfc(al * rc);
        double fc = erc / (rc * rc) + twoapi * exp(-al * al * rc * rc) / rc; /* -dV/dr of erfc(ar)/r at rc */
        double er = erfc(al * r);
        en += qq * (er / r - erc / rc + fc * (r - rc));
        f += qq * (er / (r * r) + twoapi * exp(-al * al * r * r) / r - fc);
    }
    *e = en;
    *fr = f;
}

/* Forces on the atoms listed in sel (all atoms when sel == NULL), total
 * energy and virial (sum over pairs of d (x) F, d = r_i - r_j) of one periodic
 * replica; brute force over all j and all images within rc.                   */
void ora_pair_forces(int N, const double *x, const int *type, const double box[3],
                     int ntypes, const double *charge, const double *bA, const double *brho,
                     const double *bC, double alpha, double rc, int nsel, const int *sel,
                     double *f, double *epot, double *vir)
{
    ora_pairpot pp = {ntypes, charge, bA, brho, bC, alpha, rc};
    int nmax[3];
    for (int c = 0; c < 3; ++c) nmax[c] = (int)ceil(rc / box[c]);
    double E = 0.0, W[9] = {0};
    int nloop = sel ? nsel : N;
    for (int ii = 0; ii < nloop; ++ii) {
        int i = sel ? sel[ii] : ii;
        double fi[3] = {0, 0, 0};
        for (int j = 0; j < N; ++j) {
            double d0[3];
            for (int c = 0; c < 3; ++c) {
                double d = x[3 * i + c] - x[3 * j + c];
                d0[c] = d - box[c] * round(d / box[c]);
            }
            for (int n0 = -nmax[0]; n0 <= nmax[0]; ++n0)
                for (int n1 = -nmax[1]; n1 <= nmax[1]; ++n1)
                    for (int n2 = -nmax[2]; n2 <= nmax[2]; ++n2) {
                        if (j == i && n0 == 0 && n1 == 0 && n2 == 0) continue;
                        double d[3] = {d0[0] + n0 * box[0], d0[1] + n1 * box[1], d0[2] + n2 * box[2]};
                        double r2 = d[0] * d[0] + d[1] * d[1] + d[2] * d[2];
                        if (r2 >= rc * rc) continue;
                        double r = sqrt(r2), e, fr;
                        pair_eval(&pp, type[i], type[j], r, &e, &fr);
                        for (int c = 0; c < 3; ++c) fi[c] += fr * d[c] / r;
                        E += 0.5 * e;
                        for (int a = 0; a < 3; ++a)
                            for (int b = 0; b < 3; ++b) W[3 * a + b] += 0.5 * d[a] * fr * d[b] / r;
                    }
        }
        for (int c = 0; c < 3; ++c) f[3 * ii + c] = fi[c];
    }
    if (epot) *epot = E;
    if (vir) memcpy(vir, W, sizeof W);
}

/* Separable external potentials, per Cartesian component:
 *   kind 1: V = 1/2 m w0^2 x^2        kind 2: V = V0 (x^2/a^2 - 1)^2          */
static double ext_eval(int kind, double m, double w0, double V0, double a, double x, double *fx)
{
    if (kind == 1) {
        double k = m * ORA_MVV2E * w0 * w0;
        *fx = -k * x;
        return 0.5 * k * x * x;
    }
    double u = x * x / (a * a) - 1.0;
    *fx = -4.0 * V0 * u * x / (a * a);
    return V0 * u * u;
}

/* ------------------------------------------------------------------------ */
/* Simulation state.                                                          */
typedef struct {
    int N, P, ntypes, potential, noise;
    double box[3];
    double T, gamma, dt;
    double alpha, rc;
    double ext_w0, ext_V0, ext_a;
    uint64_t seed;
    uint32_t sys;
    int32_t pad0;
    const double *mass, *charge, *bA, *brho, *bC;
    const int *type;
    const double *x0, *v0;
    int K;
    int32_t pad1;
    const double *h;
    /* isothermal-isobaric cell (npt = 1; one bead): external pressure P_ext
     * (eV/A^3), cell mass W (eV fs^2), cell friction gamma_e (1/fs) */
    int npt;
    int32_t pad2;
    double pext, wmass, gamma_e;
} ora_params;

typedef struct {
    ora_params p;
    double *mass_t, *charge_t, *bA, *brho, *bC, *h;
    int *type;
    double *x, *v, *f; /* [P][N][3] */
    double *C, *wk;
    int64_t step;
    double vsum;   /* sum over replicas of V(x_s) */
    double vir[9]; /* (1/P) sum_s W_s */
    /* white-noise window (coloured noise): win[dof*wsz + (m mod wsz)] */
    int wsz;
    double *win;
    int64_t gen_upto; /* quads generated for steps < gen_upto (multiple of 4) */
    /* isothermal-isobaric cell: momentum p_e of the log-volume / 3 and whether
     * the closing half kick of the previous step is still to be applied */
    double peps;
    int pending;
} ora_sim;

static double *dup(const double *a, size_t n)
{
    double *b = (double *)malloc(sizeof(double) * (n ? n : 1));
    if (a && n) memcpy(b, a, sizeof(double) * n);
    else if (n) memset(b, 0, sizeof(double) * n);
    return b;
}

static void compute_forces(ora_sim *s)
{
    int N = s->p.N, P = s->p.P;
    s->vsum = 0.0;
    memset(s->vir, 0, sizeof s->vir);
    for (int b = 0; b < P; ++b) {
        double *xb = s->x + (size_t)b * N * 3, *fb = s->f + (size_t)b * N * 3;
        double E = 0.0, W[9] = {0};
        if (s->p.potential == 0) {
            ora_pair_forces(N, xb, s->type, s->p.box, s->p.ntypes, s->charge_t, s->bA, s->brho,
                            s->bC, s->p.alpha, s->p.rc, 0, NULL, fb, &E, W);
        } else {
            for (int i = 0; i < N; ++i)
                for (int c = 0; c < 3; ++c) {
                    double fx;
                    E += ext_eval(s->p.potential, s->mass_t[s->type[i]], s->p.ext_w0, s->p.ext_V0,
                                  s->p.ext_a, xb[3 * i + c], &fx);
                    fb[3 * i + c] = fx;
                    W[4 * c] += xb[3 * i + c] * fx;
                }
        }
        /* Eq. 4: each bead feels -(1/P) grad V of its own replica */
        for (size_t t = 0; t < (size_t)N * 3; ++t) fb[t] /= P;
        s->vsum += E;
        for (int a = 0; a < 9; ++a) s->vir[a] += W[a] / P;
    }
}

ora_sim *ora_sim_create(const ora_params *p)
{
    ora_sim *s = (ora_sim *)calloc(1, sizeof(ora_sim));
    s->p = *p;
    int N = p->N, P = p->P, nt = p->ntypes;
    s->mass_t = dup(p->mass, nt);
    s->charge_t = dup(p->charge, nt);
    s->bA = dup(p->bA, (size_t)nt * nt);
    s->brho = dup(p->brho, (size_t)nt * nt);
    s->bC = dup(p->bC, (size_t)nt * nt);
    s->type = (int *)malloc(sizeof(int) * N);
    memcpy(s->type, p->type, sizeof(int) * N);
    s->x = dup(p->x0, (size_t)P * N * 3);
    s->v = dup(p->v0, (size_t)P * N * 3);
    s->f = dup(NULL, (size_t)P * N * 3);
    s->C = dup(NULL, (size_t)P * P);
    s->wk = dup(NULL, (size_t)P);
    ora_nm_matrix(P, s->C);
    ora_nm_freqs(P, p->T, s->wk);
    s->h = dup(p->h, p->noise ? (size_t)p->K + 1 : 0);
    s->p.mass = s->mass_t;
    s->p.charge = s->charge_t;
    s->p.bA = s->bA;
    s->p.brho = s->brho;
    s->p.bC = s->bC;
    s->p.type = s->type;
    s->p.h = s->h;
    s->p.x0 = s->p.v0 = NULL;
    if (p->noise) {
        s->wsz = 2 * p->K + 16;
        s->win = dup(NULL, (size_t)3 * N * P * s->wsz);
        s->gen_upto = 4 * quad_of(-(int64_t)p->K);
    }
    compute_forces(s);
    return s;
}

void ora_sim_destroy(ora_sim *s)
{
    if (!s) return;
    free(s->mass_t); free(s->charge_t); free(s->bA); free(s->brho); free(s->bC); free(s->h);
    free(s->type); free(s->x); free(s->v); free(s->f); free(s->C); free(s->wk); free(s->win);
    free(s);
}

/* eta for every dof at step n (coloured: filter; white: sqrt(kT) xi). */
static void noise_at(ora_sim *s, int64_t n, double *eta)
{
    int D = 3 * s->p.N * s->p.P;
    if (!s->p.noise) {
        double skT = sqrt(ORA_KB * s->p.T);
        for (int d = 0; d < D; ++d) eta[d] = skT * ora_white(s->p.seed, s->p.sys, (uint32_t)d, 0, n);
        return;
    }
    int K = s->p.K, W = s->wsz;
    while (s->gen_upto <= n + K) {
        int64_t q = quad_of(s->gen_upto);
        for (int d = 0; d < D; ++d) {
            double xi[4];
            white_quad(s->p.seed, s->p.sys, (uint32_t)d, 0, q, xi);
            for (int e = 0; e < 4; ++e) {
                int64_t m = 4 * q + e;
                int slot = (int)(((m % W) + W) % W);
                s->win[(size_t)d * W + slot] = xi[e];
            }
        }
        s->gen_upto += 4;
    }
    for (int d = 0; d < D; ++d) {
        double acc = 0.0;
        for (int k = -K; k <= K; ++k) {
            int64_t m = n - k;
            int slot = (int)(((m % W) + W) % W);
            acc += s->h[k < 0 ? -k : k] * s->win[(size_t)d * W + slot];
        }
        eta[d] = acc;
    }
}

static void observe(ora_sim *s, double *rec)
{
    int N = s->p.N, P = s->p.P;
    double K = 0.0, spring = 0.0, mom[3] = {0, 0, 0}, x2 = 0.0;
    double wP = sqrt((double)P) * ORA_KB * s->p.T / ORA_HBAR;
    for (int b = 0; b < P; ++b)
        for (int i = 0; i < N; ++i) {
            double m = s->mass_t[s->type[i]];
            int bn = (b + 1) % P;
            for (int c = 0; c < 3; ++c) {
                double vv = s->v[((size_t)b * N + i) * 3 + c];
                double xx = s->x[((size_t)b * N + i) * 3 + c];
                double dx = xx - s->x[((size_t)bn * N + i) * 3 + c];
                K += 0.5 * m * ORA_MVV2E * vv * vv;
                mom[c] += m * vv;
                spring += 0.5 * m * ORA_MVV2E * wP * wP * dx * dx;
                x2 += xx * xx;
            }
        }
    double V = s->vsum / P;
    memset(rec, 0, sizeof(double) * ORA_NREC);
    rec[0] = (double)s->step;
    rec[1] = K;
    rec[2] = V;
    rec[3] = spring;
    rec[4] = K - spring + V; /* Eq. 5, primitive estimator */
    for (int a = 0; a < 9; ++a) rec[5 + a] = s->vir[a];
    for (int c = 0; c < 3; ++c) rec[14 + c] = mom[c];
    rec[17] = x2 / P;
    rec[20] = (s->p.potential == 0) ? s->p.box[0] * s->p.box[1] * s->p.box[2] : 0.0; /* cell volume */
    /* Centroid-virial kinetic estimators.  With the bead forces f_s = -(1/P)
     * grad V(r_s) of Eq. 4 and the centroid rbar = (1/P) sum_s r_s of each atom,
     *   K_cv   = 3N k_B T/2 - 1/2 sum_i sum_s (r_i,s - rbar_i) . f_i,s
     * (PIMD: the centroid is classical at T), and, for a bath that is not
     * classical (QTB-PIMD), the same virial term with the measured kinetic
     * energy of the centroid mode, K_0 = sum_i m_i P |vbar_i|^2 / 2, in place of
     * 3N k_B T/2.  Both are exact in expectation for a harmonic potential under
     * their own bath.  Bead offsets are taken relative to bead 0, by minimum
     * image in a periodic box (the beads of an atom lie within half a box). */
    double cv = 0.0, K0 = 0.0;
    for (int i = 0; i < N; ++i) {
        double m = s->mass_t[s->type[i]];
        for (int c = 0; c < 3; ++c) {
            double L = (s->p.potential == 0) ? s->p.box[c] : 0.0;
            double x0 = s->x[(size_t)i * 3 + c];
            double dbar = 0.0, vs = 0.0;
            for (int b = 0; b < P; ++b) {
                double d = s->x[((size_t)b * N + i) * 3 + c] - x0;
                if (L > 0.0) d -= L * round(d / L);
                dbar += d;
                vs += s->v[((size_t)b * N + i) * 3 + c];
            }
            dbar /= P;
            for (int b = 0; b < P; ++b) {
                double d = s->x[((size_t)b * N + i) * 3 + c] - x0;
                if (L > 0.0) d -= L * round(d / L);
                cv += (d - dbar) * s->f[((size_t)b * N + i) * 3 + c];
            }
            K0 += 0.5 * m * ORA_MVV2E * vs * vs / P;
        }
    }
    rec[18] = 1.5 * N * ORA_KB * s->p.T - 0.5 * cv;
    rec[19] = K0 - 0.5 * cv;
    /* the centroid modes' kinetic energy and the centroid virial (trace): the
     * cell's generalised force of an isothermal-isobaric run (for one bead K
     * and the virial trace) */
    rec[21] = K0;
    rec[22] = (s->vir[0] + s->vir[4] + s->vir[8]) - cv;
}

/* ------------------------------------------------------------------------ */
/* Isothermal-isobaric step (one bead, pair potential; ring polymers below): the equations and the
 * splitting are in the header comment.  Positions are physical (A); the cell
 * edges scale by exp(v_e t).                                                   */
static double kinetic(const ora_sim *s)
{
    double K = 0.0;
    for (int i = 0; i < s->p.N; ++i)
        for (int c = 0; c < 3; ++c) {
            double v = s->v[(size_t)i * 3 + c];
            K += 0.5 * s->mass_t[s->type[i]] * ORA_MVV2E * v * v;
        }
    return K;
}

/* dG: the cell's generalised force 2 alpha K + Wvir - 3 V P_ext */
static double cell_force(const ora_sim *s, double alpha)
{
    double V = s->p.box[0] * s->p.box[1] * s->p.box[2];
    double wvir = s->vir[0] + s->vir[4] + s->vir[8];
    return 2.0 * alpha * kinetic(s) + wvir - 3.0 * V * s->p.pext;
}

/* B(dt/2): exact solution of dv/dt = F/m - alpha v_e v */
static void kick_npt(ora_sim *s, double alpha, double ve, double h)
{
    double x = alpha * ve * h;
    double e = exp(-x);
    double g = (x != 0.0) ? -expm1(-x) / x : 1.0; /* (1 - e^{-x}) / x */
    for (int i = 0; i < s->p.N; ++i) {
        double m = s->mass_t[s->type[i]] * ORA_MVV2E;
        for (int c = 0; c < 3; ++c) {
            size_t k = (size_t)i * 3 + c;
            s->v[k] = s->v[k] * e + h * s->f[k] / m * g;
        }
    }
}

/* A(dt/2): exact solution of dr/dt = v + v_e r, the cell edges scaled alike */
static void drift_npt(ora_sim *s, double ve, double h)
{
    double x = ve * h;
    double e = exp(x);
    double g = (x != 0.0) ? expm1(x) / x : 1.0; /* (e^{x} - 1) / x */
    for (size_t k = 0; k < (size_t)s->p.N * 3; ++k) s->x[k] = s->x[k] * e + s->v[k] * h * g;
    for (int c = 0; c < 3; ++c) s->p.box[c] *= e;
}

static void step_npt(ora_sim *s, double *rec1)
{
    int N = s->p.N, D = 3 * N;
    double dt = s->p.dt, h = 0.5 * dt;
    double c1 = exp(-s->p.gamma * dt), ce = exp(-s->p.gamma_e * dt);
    double alpha = 1.0 + 3.0 / (3.0 * N);
    double W = s->p.wmass;
    double *eta = dup(NULL, (size_t)D);
    int64_t n = s->step;
    noise_at(s, n, eta);
    /* B_e(dt/2): the closing half of the previous step (if any), then this one */
    double G = cell_force(s, alpha);
    if (s->pending) s->peps += h * G;
    s->peps += h * G;
    double ve = s->peps / W;
    kick_npt(s, alpha, ve, h);  /* B */
    drift_npt(s, ve, h);        /* A */
    for (int i = 0; i < N; ++i) { /* O, particles */
        double m = s->mass_t[s->type[i]] * ORA_MVV2E;
        double sig = sqrt((1.0 - c1 * c1) / m);
        for (int c = 0; c < 3; ++c) {
            size_t k = (size_t)i * 3 + c;
            s->v[k] = c1 * s->v[k] + sig * eta[(size_t)c * N + i];
        }
    }
    /* O, cell: white noise at k_B T, Philox stream 1, dof 0 */
    double xi = ora_white(s->p.seed, s->p.sys, 0u, 1u, n);
    s->peps = ce * s->peps + sqrt((1.0 - ce * ce) * W * ORA_KB * s->p.T) * xi;
    ve = s->peps / W;
    drift_npt(s, ve, h);        /* A */
    compute_forces(s);
    kick_npt(s, alpha, ve, h);  /* B; B_e(dt/2) closes at the next step */
    s->pending = 1;
    s->step += 1;
    if (rec1) observe(s, rec1);
    free(eta);
}

/* Ring polymers at constant pressure: K_0 and sum_i sum_s (r_i,s - rbar_i) .
 * f_i,s, bead offsets by minimum image about bead 0 (as in observe). */
static void centroid_terms(const ora_sim *s, double *K0_out, double *cv_out)
{
    int N = s->p.N, P = s->p.P;
    double cv = 0.0, K0 = 0.0;
    for (int i = 0; i < N; ++i) {
        double m = s->mass_t[s->type[i]];
        for (int c = 0; c < 3; ++c) {
            double L = s->p.box[c];
            double x0 = s->x[(size_t)i * 3 + c];
            double dbar = 0.0, vs = 0.0;
            for (int b = 0; b < P; ++b) {
                double d = s->x[((size_t)b * N + i) * 3 + c] - x0;
                d -= L * round(d / L);
                dbar += d;
                vs += s->v[((size_t)b * N + i) * 3 + c];
            }
            dbar /= P;
            for (int b = 0; b < P; ++b) {
                double d = s->x[((size_t)b * N + i) * 3 + c] - x0;
                d -= L * round(d / L);
                cv += (d - dbar) * s->f[((size_t)b * N + i) * 3 + c];
            }
            K0 += 0.5 * m * ORA_MVV2E * vs * vs / P;
        }
    }
    *K0_out = K0;
    *cv_out = cv;
}

/* modes of one atom-component: out[k] = sum_b C[b][k] a[b, i, c] */
static void to_modes(const ora_sim *s, const double *a, int i, int c, double *out)
{
    int N = s->p.N, P = s->p.P;
    for (int k = 0; k < P; ++k) {
        double acc = 0.0;
        for (int b = 0; b < P; ++b) acc += s->C[b * P + k] * a[((size_t)b * N + i) * 3 + c];
        out[k] = acc;
    }
}

static void to_beads(const ora_sim *s, const double *m, int i, int c, double *a)
{
    int N = s->p.N, P = s->p.P;
    for (int b = 0; b < P; ++b) {
        double acc = 0.0;
        for (int k = 0; k < P; ++k) acc += s->C[b * P + k] * m[k];
        a[((size_t)b * N + i) * 3 + c] = acc;
    }
}

/* The ring-polymer isothermal-isobaric step (P > 1; equations in the header
 * comment).  Positions are physical and unwrapped; the centroid mode Q_0 drifts
 * as dQ_0/dt = p_0 + v_e Q_0, the internal modes rotate freely. */
static void step_npt_rp(ora_sim *s, double *rec1)
{
    int N = s->p.N, P = s->p.P, D = 3 * N * P;
    double dt = s->p.dt, h = 0.5 * dt;
    double c1 = exp(-s->p.gamma * dt), ce = exp(-s->p.gamma_e * dt);
    double alpha = 1.0 + 3.0 / (3.0 * N);
    double W = s->p.wmass;
    double *eta = dup(NULL, (size_t)D), *q = dup(NULL, (size_t)P), *pm = dup(NULL, (size_t)P),
           *fk = dup(NULL, (size_t)P);
    int64_t n = s->step;
    noise_at(s, n, eta);
    /* B_e(dt/2) twice (the first closes the previous step), from K_0 and W_cv */
    double K0, cv;
    centroid_terms(s, &K0, &cv);
    double Vol = s->p.box[0] * s->p.box[1] * s->p.box[2];
    double G = 2.0 * alpha * K0 + ((s->vir[0] + s->vir[4] + s->vir[8]) - cv) - 3.0 * Vol * s->p.pext;
    if (s->pending) s->peps += h * G;
    s->peps += h * G;
    double ve1 = s->peps / W;
    /* O of the cell (between the two A halves; independent of the particles) */
    double xi = ora_white(s->p.seed, s->p.sys, 0u, 1u, n);
    double peps2 = ce * s->peps + sqrt((1.0 - ce * ce) * W * ORA_KB * s->p.T) * xi;
    double ve2 = peps2 / W;
    double x1 = alpha * ve1 * h, e1 = exp(-x1), g1 = (x1 != 0.0) ? -expm1(-x1) / x1 : 1.0;
    double y1 = ve1 * h, ey1 = exp(y1), gy1 = (y1 != 0.0) ? expm1(y1) / y1 : 1.0;
    double y2 = ve2 * h, ey2 = exp(y2), gy2 = (y2 != 0.0) ? expm1(y2) / y2 : 1.0;
    for (int i = 0; i < N; ++i) {
        double m = s->mass_t[s->type[i]] * ORA_MVV2E;
        double sig = sqrt((1.0 - c1 * c1) / m);
        for (int c = 0; c < 3; ++c) {
            to_modes(s, s->x, i, c, q);
            to_modes(s, s->v, i, c, pm);
            to_modes(s, s->f, i, c, fk);
            /* B(dt/2): the centroid with the cell's friction */
            pm[0] = pm[0] * e1 + h * fk[0] / m * g1;
            for (int k = 1; k < P; ++k) pm[k] += h * fk[k] / m;
            for (int half = 0; half < 2; ++half) {
                /* A(dt/2): centroid drift with the cell, internal modes rotate */
                double ey = half ? ey2 : ey1, gy = half ? gy2 : gy1;
                q[0] = q[0] * ey + pm[0] * h * gy;
                for (int k = 1; k < P; ++k) {
                    double w = s->wk[k];
                    double cs = cos(h * w), sn = sin(h * w);
                    double qn = q[k] * cs + pm[k] / w * sn;
                    double pn = -q[k] * w * sn + pm[k] * cs;
                    q[k] = qn;
                    pm[k] = pn;
                }
                if (half == 0) /* O(dt), every mode */
                    for (int k = 0; k < P; ++k) pm[k] = c1 * pm[k] + sig * eta[(size_t)(k * 3 + c) * N + i];
            }
            to_beads(s, q, i, c, s->x);
            to_beads(s, pm, i, c, s->v);
        }
    }
    for (int c = 0; c < 3; ++c) {
        s->p.box[c] *= ey1;
        s->p.box[c] *= ey2;
    }
    s->peps = peps2;
    compute_forces(s);
    /* closing B(dt/2) with the new v_e */
    double x2 = alpha * ve2 * h, e2 = exp(-x2), g2 = (x2 != 0.0) ? -expm1(-x2) / x2 : 1.0;
    for (int i = 0; i < N; ++i) {
        double m = s->mass_t[s->type[i]] * ORA_MVV2E;
        for (int c = 0; c < 3; ++c) {
            to_modes(s, s->v, i, c, pm);
            to_modes(s, s->f, i, c, fk);
            pm[0] = pm[0] * e2 + h * fk[0] / m * g2;
            for (int k = 1; k < P; ++k) pm[k] += h * fk[k] / m;
            to_beads(s, pm, i, c, s->v);
        }
    }
    s->pending = 1;
    s->step += 1;
    if (rec1) observe(s, rec1);
    free(eta); free(q); free(pm); free(fk);
}

/* Advance nsteps BAOAB steps; if rec != NULL write one record per step. */
void ora_sim_step(ora_sim *s, int64_t nsteps, double *rec)
{
    if (s->p.npt) {
        for (int64_t it = 0; it < nsteps; ++it) {
            double *r1 = rec ? rec + (size_t)it * ORA_NREC : NULL;
            if (s->p.P == 1) step_npt(s, r1);
            else step_npt_rp(s, r1);
        }
        return;
    }
    int N = s->p.N, P = s->p.P, D = 3 * N * P;
    double dt = s->p.dt;
    double c1 = exp(-s->p.gamma * dt);
    double *eta = dup(NULL, (size_t)D), *q = dup(NULL, (size_t)P), *pm = dup(NULL, (size_t)P);
    for (int64_t it = 0; it < nsteps; ++it) {
        int64_t n = s->step;
        noise_at(s, n, eta);
        /* B: half kick in bead space */
        for (int b = 0; b < P; ++b)
            for (int i = 0; i < N; ++i) {
                double m = s->mass_t[s->type[i]] * ORA_MVV2E;
                for (int c = 0; c < 3; ++c) {
                    size_t g = ((size_t)b * N + i) * 3 + c;
                    s->v[g] += 0.5 * dt * s->f[g] / m;
                }
            }
        /* A O A in normal-mode space, per atom and Cartesian component */
        for (int i = 0; i < N; ++i) {
            double m = s->mass_t[s->type[i]] * ORA_MVV2E;
            double sig = sqrt((1.0 - c1 * c1) / m);
            for (int c = 0; c < 3; ++c) {
                for (int k = 0; k < P; ++k) {
                    double a = 0.0, bb = 0.0;
                    for (int b = 0; b < P; ++b) {
                        a += s->C[b * P + k] * s->x[((size_t)b * N + i) * 3 + c];
                        bb += s->C[b * P + k] * s->v[((size_t)b * N + i) * 3 + c];
                    }
                    q[k] = a;
                    pm[k] = bb;
                }
                for (int half = 0; half < 2; ++half) {
                    for (int k = 0; k < P; ++k) {
                        double w = s->wk[k];
                        if (w == 0.0) {
                            q[k] += 0.5 * dt * pm[k];
                        } else {
                            double cs = cos(0.5 * dt * w), sn = sin(0.5 * dt * w);
                            double qn = q[k] * cs + pm[k] / w * sn;
                            double pn = -q[k] * w * sn + pm[k] * cs;
                            q[k] = qn;
                            pm[k] = pn;
                        }
                    }
                    if (half == 0)
                        for (int k = 0; k < P; ++k)
                            pm[k] = c1 * pm[k] + sig * eta[(size_t)(k * 3 + c) * N + i];
                }
                for (int b = 0; b < P; ++b) {
                    double a = 0.0, bb = 0.0;
                    for (int k = 0; k < P; ++k) {
                        a += s->C[b * P + k] * q[k];
                        bb += s->C[b * P + k] * pm[k];
                    }
                    s->x[((size_t)b * N + i) * 3 + c] = a;
                    s->v[((size_t)b * N + i) * 3 + c] = bb;
                }
            }
        }
        compute_forces(s);
        for (int b = 0; b < P; ++b)
            for (int i = 0; i < N; ++i) {
                double m = s->mass_t[s->type[i]] * ORA_MVV2E;
                for (int c = 0; c < 3; ++c) {
                    size_t g = ((size_t)b * N + i) * 3 + c;
                    s->v[g] += 0.5 * dt * s->f[g] / m;
                }
            }
        s->step += 1;
        if (rec) observe(s, rec + (size_t)it * ORA_NREC);
    }
    free(eta); free(q); free(pm);
}

void ora_sim_observe(ora_sim *s, double *rec) { observe(s, rec); }

void ora_sim_get(const ora_sim *s, double *x, double *v, double *f, int64_t *step)
{
    size_t n = (size_t)s->p.P * s->p.N * 3;
    if (x) memcpy(x, s->x, sizeof(double) * n);
    if (v) memcpy(v, s->v, sizeof(double) * n);
    if (f) memcpy(f, s->f, sizeof(double) * n);
    if (step) *step = s->step;
}

/* Replace positions/velocities (and the step index) and recompute forces. */
void ora_sim_set(ora_sim *s, const double *x, const double *v, int64_t step)
{
    size_t n = (size_t)s->p.P * s->p.N * 3;
    if (x) memcpy(s->x, x, sizeof(double) * n);
    if (v) memcpy(s->v, v, sizeof(double) * n);
    if (step != s->step && s->p.noise) s->gen_upto = 4 * quad_of(step - (int64_t)s->p.K);
    s->step = step;
    compute_forces(s);
}

int ora_nrec(void) { return ORA_NREC; }

/* Replace the cell of an isothermal-isobaric run (edges, momentum, whether the
 * previous step's closing half kick is due) and recompute the forces. */
void ora_sim_set_cell(ora_sim *s, const double *box, double peps, int pending)
{
    memcpy(s->p.box, box, sizeof(double) * 3);
    s->peps = peps;
    s->pending = pending;
    compute_forces(s);
}

/* Cell edges (A) and cell momentum p_e of an isothermal-isobaric run. */
void ora_sim_cell(const ora_sim *s, double *box, double *peps)
{
    if (box) memcpy(box, s->p.box, sizeof(double) * 3);
    if (peps) *peps = s->peps;
}
