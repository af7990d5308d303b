/*
 * qtb.h -- C ABI of the GB300 quantum-thermal-bath molecular-dynamics hot path.
 *
 * Method: Dammak, Hayoun, Brieuc, Geneste, "Nuclear quantum effects in molecular
 * dynamics simulations".  The library advances one or many independent systems
 * (atoms x ring-polymer beads) with a Langevin (BAOAB) integrator whose random
 * force is coloured so that its power spectral density is 2 m gamma theta(w,T)
 * (Eqs. 6-8, QTB-MD) or 2 m gamma kappa_P(w,T) applied to the ring-polymer
 * normal modes (Eqs. 10-12, QTB-PIMD), or white (classical Langevin / PIMD).
 *
 * Conventions
 *   units       A, fs, eV, u (atomic mass), e, K; frequencies in rad/fs.
 *   errors      every call returns a qtb_status (0 = QTB_OK, negative = error);
 *               qtb_last_error() gives a one-line message.  No exception or
 *               longjmp crosses this boundary.
 *   host arrays are borrowed for the duration of the call only (copied).
 *   device memory is owned by the library; it is obtained through the
 *               caller's allocator callbacks when given (e.g. a PyTorch caching
 *               allocator), else cudaMalloc.
 *   streams     all device work is issued on the stream given to qtb_init
 *               (NULL: the library creates and owns a non-blocking stream).  qtb_step_n is asynchronous;
 *               qtb_observables, qtb_get_* and qtb_sync synchronise the stream
 *               and report device-side errors (cell overflow, non-finite
 *               state) raised by earlier steps.
 *   threads     a context must not be used from two threads at once.
 */
#ifndef QTB_H
#define QTB_H

#include <stddef.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct qtb_ctx qtb_ctx; /* opaque, owned by the library */

typedef enum {
    QTB_OK = 0,
    QTB_ERR_ARG = -1,       /* invalid argument (message says which)           */
    QTB_ERR_CUDA = -2,      /* a CUDA runtime/driver call failed                */
    QTB_ERR_OOM = -3,       /* device allocation failed                         */
    QTB_ERR_TIMEOUT = -4,   /* a bounded device wait gave up (barrier, mbarrier) */
    QTB_ERR_NONFINITE = -5, /* a force or velocity became NaN/Inf               */
    QTB_ERR_SOLVE = -6,     /* kappa_P solve failed (non-positive pivot or PSD) */
    QTB_ERR_OVERFLOW = -7,  /* a cell or a neighbour list overflowed its capacity */
    QTB_ERR_STATE = -8      /* call not valid in the current state              */
} qtb_status;

/* Arithmetic of the step.  QTB_FP64: every step in FP64.  QTB_MIXED: positions
 * in 30-bit fixed point per box length, forces/integration in FP32, energies
 * and virials accumulated in FP64, noise filter per qtb_filter_prec. */
typedef enum { QTB_FP64 = 0, QTB_MIXED = 1 } qtb_precision;

/* Noise filter arithmetic (QTB_MIXED only; QTB_FP64 always filters in FP64).
 * FP32: direct FP32 convolution.  BF16: blocked Toeplitz GEMM on the tensor
 * cores (tcgen05, BF16 operands, FP32 accumulation). */
typedef enum { QTB_FILTER_FP64 = 0, QTB_FILTER_FP32 = 1, QTB_FILTER_BF16 = 2 } qtb_filter_prec;

/* Random force of the O step.
 *   WHITE    classical Langevin (PIMD when n_beads > 1): PSD 2 m gamma k_B T.
 *   QTB      PSD 2 m gamma theta(w,T), Eq. 7 (n_beads must be 1).
 *   QTB_PIMD PSD 2 m gamma kappa_P(w,T) per normal mode, Eq. 12.
 *   QTB_PIMD_MLP as QTB_PIMD with kappa_P from the learned model set by
 *            qtb_set_kappa_model (falls back to the solver where the model's
 *            error, judged by the solver, exceeds its tolerance). */
typedef enum { QTB_NOISE_WHITE = 0, QTB_NOISE_QTB = 1, QTB_NOISE_QTB_PIMD = 2, QTB_NOISE_QTB_PIMD_MLP = 3 } qtb_noise;

/* Potential energy surface.  PAIR: Buckingham (energy-shifted at r_cut) plus
 * damped-shifted-force Coulomb (Fennell & Gezelter 2006) in an orthorhombic
 * periodic box, all images within r_cut.  HARMONIC / DOUBLEWELL: separable
 * external potential per Cartesian component, 1/2 m w0^2 x^2 or
 * V0 (x^2/a^2 - 1)^2 (no box). */
typedef enum { QTB_POT_PAIR = 0, QTB_POT_HARMONIC = 1, QTB_POT_DOUBLEWELL = 2 } qtb_potential;

typedef struct {
    int n_atoms;        /* N >= 1                                                  */
    int n_beads;        /* P in {1..6, 8, 16, 32} (Trotter number of Eq. 2)      */
    const int *type;    /* [N] type index < n_types                               */
    const double *pos;  /* [P][N][3] bead positions, A                             */
    const double *vel;  /* [P][N][3] bead velocities, A/fs; NULL = zero           */
    double box[3];      /* orthorhombic box edges, A (PAIR only; each >= r_cut)   */
    double T;           /* temperature, K (> 0)                                    */
    double gamma;       /* friction coefficient of Eq. 8, 1/fs (>= 0)             */
} qtb_system;

typedef void *(*qtb_alloc_fn)(size_t bytes, void *user);
typedef void (*qtb_free_fn)(void *ptr, void *user);

typedef struct {
    int n_types;
    const double *mass;    /* [n_types] u                                          */
    const double *charge;  /* [n_types] e                                          */
    const double *buck_A;  /* [n_types*n_types] eV   (0 = no Buckingham term)      */
    const double *buck_rho;/* [n_types*n_types] A                                  */
    const double *buck_C;  /* [n_types*n_types] eV A^6                              */
    double dsf_alpha;      /* DSF damping, 1/A                                     */
    double r_cut;          /* cutoff, A                                            */
    int potential;         /* qtb_potential                                        */
    double ext_omega;      /* HARMONIC: w0, rad/fs                                 */
    double ext_V0, ext_a;  /* DOUBLEWELL: V0 (eV), a (A)                           */
    double dt;             /* time step, fs                                        */
    int precision;         /* qtb_precision                                        */
    int filter_prec;       /* qtb_filter_prec                                      */
    unsigned long long seed; /* Philox key; system s uses key (lo32(seed), hi32(seed)^s) */
    int obs_stride;        /* record observables every obs_stride steps (>= 1)     */
    int max_records;       /* capacity of the per-system observable series (>= 1)  */
    qtb_alloc_fn dev_alloc;  /* optional device allocator                          */
    qtb_free_fn dev_free;    /* its matching free                                  */
    void *alloc_user;        /* passed to both                                     */
    double skin;           /* PAIR: Verlet-list skin, A, < r_cut/2.  Lists hold every
                              pair within r_cut + skin and are rebuilt (on the device)
                              once some bead-atom has moved skin/2 since the last
                              rebuild.  0 selects, per system, min(r_cut/4,
                              0.8 max(1, sqrt(T/300 K))) (hot systems move further
                              between rebuilds); < 0: no skin.
                              Forces do not depend on it (up to summation order). */
    int nm_layout;         /* ring-polymer integrator (n_beads > 1): 0 auto, 1 compact
                              (8-32 atoms per CTA, more CTAs; small contexts), 2 wide (32
                              atoms per CTA, coalesced rows; large contexts).  Same
                              arithmetic, bit-identical results. */
    int list_lanes;        /* PAIR: lanes per bead-atom of the force kernel, 8, 16 or 32
                              (0: 16).  Changes the summation order only. */
    int rebuild_scope;     /* PAIR: 0 a list rebuild covers the systems one of whose
                              bead-atoms moved skin/2 (each system of a batch then runs
                              bit for bit as it would alone); 1 every system of the
                              context (fewer, larger rebuilds for batches of hot and
                              cold systems; results change at the rounding level). */
    /* Isothermal-isobaric runs (Sec. 2.1: the paper's constant-pressure
     * simulations use Quigley and Probert's Langevin extension, refs [11, 12];
     * it prints no equations).  npt = 1: every system's cell is an isotropic
     * Langevin barostat, the isotropic Martyna-Tobias-Klein equations with
     * friction and noise on the particles and on the cell:
     *   dr/dt = v + v_e r,  m dv/dt = F - (1 + 3/N_f) m v_e v - gamma m v + R,
     *   dV/dt = 3 V v_e,    dp_e/dt = 2 (1 + 3/N_f) K + W_vir - 3 V P_ext
     *                                 - cell_gamma p_e + R_e,   v_e = p_e / cell_mass,
     * N_f = 3N, W_vir the pair virial; R the particle random force of the chosen
     * noise (QTB: Eq. 7), R_e white at k_B T.  Stationary law:
     * P(V) ~ V^N exp(-(U + P_ext V)/k_B T) for the white bath.  Ring polymers
     * (P > 1): the cell acts on each atom's centroid mode (sqrt(P) rbar) only,
     * the bead offsets from the centroid are physical and do not scale with it;
     * K and W_vir above become the centroid modes' kinetic energy K_0 and the
     * centroid virial W_cv (record slots 21 and 22).  Pair potential only; the
     * cell may shrink to 0.9 of its initial edges (QTB_ERR_STATE below that: the
     * cell lists keep that margin). */
    int npt;               /* 0: constant volume; 1: isotropic Langevin barostat        */
    double pressure;       /* P_ext, eV/A^3 (1 GPa = 6.241509e-3 eV/A^3)                */
    double cell_mass;      /* W, eV fs^2 (> 0)                                          */
    double cell_gamma;     /* friction of the cell, 1/fs (>= 0)                          */
} qtb_params;

/* Observable record (FP64), one per recorded step and system:
 *   [0] step index after the step   [1] K = sum 1/2 m v^2 over beads (eV)
 *   [2] V = (1/P) sum_s V(r^(s))    [3] spring = sum_s sum_i 1/2 m w_P^2 (r_s - r_{s+1})^2
 *   [4] E_prim = K - spring + V (Eq. 5)
 *   [5..13] virial (1/P) sum_s sum_pairs d (x) F, row-major 3x3 (eV)
 *   [14..16] total momentum (u A/fs)   [17] (1/P) sum_s sum_i |r_i^(s)|^2 (A^2)
 *   [18] K_cv = 3N k_B T/2 - 1/2 sum_s sum_i (r_i^(s) - rbar_i) . f_i^(s), the
 *        centroid-virial kinetic energy (f = -(1/P) grad V, Eq. 4; rbar the bead
 *        centroid, bead offsets by minimum image); PIMD, classical centroid
 *   [19] K_cv,0: the same with 3N k_B T/2 replaced by the centroid-mode kinetic
 *        energy sum_i m_i P |vbar_i|^2/2 (a bath that does not hold the centroid
 *        at k_B T: QTB-PIMD).  The paper prints neither (only Eq. 5).  One
 *        bead: [18] = 3N k_B T/2, [19] = K.
 *   [20] cell volume (A^3; constant unless npt; 0 for external potentials)
 *   [21] K_0 = sum_i m_i P |vbar_i|^2/2, the centroid modes' kinetic energy
 *   [22] W_cv = (1/P) sum_s W_vir,s - sum_s sum_i (r_i^(s) - rbar_i) . f_i^(s),
 *        the centroid virial (trace): the virial of a scaling of the centroids
 *        at fixed bead offsets.  One bead: [21] = K, [22] = the virial trace.
 *        [21] and [22] of ring polymers, like [18] and [19], are formed on
 *        recorded steps (every step at constant pressure). */
#define QTB_NREC 23

/* Create a context for n_sys independent systems sharing one parameter set.
 * Copies the host arrays, allocates device state, computes the first forces.
 * The noise starts WHITE for every system (call qtb_set_filter to change).
 * Reads: Eqs. 3-4 (ring polymer), Eq. 8 (Langevin).  stream: a cudaStream_t. */
int qtb_init(qtb_ctx **out, const qtb_system *sys, int n_sys, const qtb_params *p, void *stream);

/* Choose the random force of system sys (-1 = all systems).
 * mode: qtb_noise.  n_taps: odd filter length L = 2K+1 of the zero-phase
 * time-domain filter (ignored for WHITE).  omega_max: Fermi cutoff of the
 * spectrum, rad/fs (<= 0: none).  Builds theta(w_j,T) (Eq. 1) or kappa_P
 * (Eq. 10, solved in FP64 on the GPU) on w_j = 2 pi j/(L dt), then the taps by
 * an FP64 cosine transform.  Takes effect from the next step; the stochastic
 * trajectory for a given seed does not depend on when it is called, only on
 * the filter in force at each step. */
int qtb_set_filter(qtb_ctx *c, int sys, int mode, int n_taps, double omega_max);

/* Generator of the coloured noise, for every system of the context.
 *   QTB_GEN_FILTER  (default) the zero-phase time-domain filter of qtb_set_filter:
 *                   stationary noise, no segment boundaries.
 *   QTB_GEN_FOURIER the paper's own method (Eq. 9, Sec. 2.2): segments of
 *                   n = 256 segment_blocks steps (segment_blocks in {1, 2, 4, 8}),
 *                   each drawn in Fourier space on w_j = 2 pi j/(n dt) from the
 *                   n normals of the white stream over the segment and brought to
 *                   the time domain by an inverse FFT; discrete spectral density
 *                   S = theta W (kappa_P W for QTB-PIMD, k_B T for WHITE), the
 *                   mode and cutoff of qtb_set_filter (n_taps unused).  The noise
 *                   is periodic within a segment and uncorrelated across segments.
 * The learned kappa_P mode is not available with QTB_GEN_FOURIER (QTB_ERR_ARG).
 * Takes effect from the next step. */
typedef enum { QTB_GEN_FILTER = 0, QTB_GEN_FOURIER = 1 } qtb_generator;
int qtb_set_generator(qtb_ctx *c, int generator, int segment_blocks);

/* Advance every system by n_steps steps of the Langevin equation of motion
 * (asynchronous): Eq. 8 for one bead (QTB-MD, the random force of Eqs. 6-7) and
 * Eq. 4 with the ring-polymer springs of Eq. 3 for P beads (PIMD; QTB-PIMD
 * with the random force of Eq. 12 on the normal modes of Eq. 11).  The paper
 * does not fix the integrator; the reading used is BAOAB: a half kick by the
 * forces (B), the exact free ring-polymer motion for dt/2 per normal mode (A),
 * the friction and random force over dt (O: v <- c1 v + sqrt((1 - c1^2)/m) eta,
 * c1 = exp(-gamma dt)), A, new forces, B.  With qtb_params.npt the cell's
 * equations (given there) join every step.  Whole 256-step noise blocks run as
 * one CUDA-graph launch.  n_steps >= 0 (0: no-op). */
int qtb_step_n(qtb_ctx *c, long long n_steps);

/* Wait for the stream; report device-side errors of earlier steps. */
int qtb_sync(qtb_ctx *c);

/* Latest observable record of system sys (QTB_NREC doubles, host; layout
 * above): the kinetic and potential energies and the primitive energy
 * estimator of Eq. 5 (E = K - spring + V, with the spring term of Eq. 3 and
 * V/P per replica of Eq. 4), the virial, the total momentum, the mean square
 * position, the centroid-virial kinetic estimators, the cell volume and the
 * centroid kinetic energy and virial.  Synchronises once; returns a device-side
 * error of an earlier step if one was raised (out is then filled as it is). */
int qtb_observables(qtb_ctx *c, int sys, double *out);

/* All records kept for system sys, oldest first: out[max][QTB_NREC]; *n_out =
 * number written (at most max_records of qtb_params). */
int qtb_get_series(qtb_ctx *c, int sys, double *out, int max, int *n_out);

/* Bead positions/velocities [P][N][3] of system sys (host FP64).  Positions
 * are wrapped into the box for PAIR systems.  Either pointer may be NULL. */
int qtb_get_state(qtb_ctx *c, int sys, double *pos, double *vel);

/* Replace positions/velocities of system sys (either may be NULL = keep).  The
 * forces and the observable record at the current step index are recomputed
 * once, at the next call that needs them (qtb_step_n, qtb_sync,
 * qtb_observables, qtb_get_series, qtb_get_state, qtb_get_forces,
 * qtb_list_rebuilds), so that setting several systems costs one force
 * evaluation; an error of that evaluation is returned by that call.  PAIR:
 * positions may lie in any periodic image (each is taken modulo the box, as the
 * copy nearest its position at the last list rebuild, so the state that
 * qtb_get_state reports goes back unchanged); a system's neighbour lists are
 * rebuilt then only if one of its bead-atoms lies more than skin/2 from its
 * position at the last rebuild (the criterion of the steps); otherwise they
 * stay valid and are kept. */
int qtb_set_state(qtb_ctx *c, int sys, const double *pos, const double *vel);

/* Forces [P][N][3] (eV/A) of system sys at the current positions, including the
 * 1/P factor of Eq. 4. */
int qtb_get_forces(qtb_ctx *c, int sys, double *f);

/* Filter taps h_0..h_K (FP64) of system sys; *n_out = K+1. */
int qtb_get_taps(qtb_ctx *c, int sys, double *h, int max, int *n_out);

/* Coloured noise eta (the O step uses sqrt((1-c1^2)/m) eta) for the 256-step
 * block containing the current step, system sys: out[256][3 N P] (FP64),
 * dof = (mode k * 3 + component) * N + atom; *block_out = block index. */
int qtb_get_noise(qtb_ctx *c, int sys, double *out, long long *block_out);

/* Profiling of whole 256-step blocks: when enabled, the captured block records
 * a CUDA event pair around the launches of every 64th step and around the
 * per-block noise launches (classes: 0 white noise, 1 filter, 2 integrator,
 * 3 unused (list rebuilds run inside the force launch), 4 force (pair
 * potential: the step kernel, with a list rebuild when one is due and, for
 * one-bead systems, the first half of the next step), 5 reduction).  Takes
 * effect at the next block. */
int qtb_set_profiling(qtb_ctx *c, int enable);

/* Mean device time (ms) and launch count per kernel class over the last
 * profiled block (synchronises).  mean_ms, counts: [n_classes]. */
int qtb_kernel_times(qtb_ctx *c, double *mean_ms, int *counts, int n_classes);

/* Number of neighbour-list rebuilds carried out so far (PAIR; 0 otherwise),
 * the one made by qtb_init included (and those an uploaded state needed; see
 * qtb_set_state).  Synchronises. */
int qtb_list_rebuilds(qtb_ctx *c, long long *count);

/* Rebuild the neighbour lists of every system (PAIR; a no-op otherwise) on the
 * current positions, at the next call that needs the forces (as after
 * qtb_set_state); the forces and the record of the current step are evaluated
 * again.  Changes no state: lists are otherwise rebuilt only when a bead-atom
 * has moved skin/2.  Use: lists built on the initial, nearly perfect lattice
 * hold the same number of entries for every ion and are traversed faster than
 * any later lists; rebuilding them on a thermalised configuration gives the
 * steady state of a long trajectory.  No counterpart in the paper. */
int qtb_rebuild_lists(qtb_ctx *c);

/* Self-test of the device's bounded waits (no counterpart in the paper; the
 * grid barriers of the step kernel and the list rebuild use them).  One device
 * thread waits, through the same bounded wait, on a flag that nothing sets; the
 * wait gives up after about one second of device time and records that in a
 * status word of its own, not in the context's error word, so the context stays
 * usable.  Outputs: *gave_up = 1 when the wait gave up (the expected outcome),
 * *ms = the kernel's duration.  Returns QTB_OK when the kernel ran.
 * Synchronises. */
int qtb_wait_selftest(qtb_ctx *c, int *gave_up, double *ms);

/* Result of qtb_autotune. */
typedef struct {
    double skin;          /* chosen neighbour-list skin, A (0: the default) */
    int nm_layout;        /* chosen ring-polymer integrator layout (1 compact, 2 wide; 0 if P = 1 only) */
    int list_lanes;       /* chosen lanes per bead-atom of the force kernel (0: the default, 16) */
    int rebuild_scope;    /* chosen rebuild scope (0 requesting systems, 1 all; 0 for one system) */
    double ms_per_step;   /* mean device time of one MD step with that choice */
    double default_ms_per_step;  /* the same with the defaults (skin 0, nm_layout 0, list_lanes 0,
                                    rebuild_scope 0) */
    int n_tried;          /* configurations timed */
} qtb_tuning;

/* Autotuner of the launch shapes and the cell/neighbour-list batching.  For
 * every candidate -- skin in {0.5, 0.8, 1.2, 1.6} A (those below r_cut/2),
 * lanes per bead-atom in {8, 16, 32}, for systems with beads the integrator
 * layouts {1, 2}, and for several systems the rebuild scopes {0, 1} -- it creates a context for the given systems and parameters
 * (qtb_init), applies the filter (noise_mode, n_taps, omega_max; as
 * qtb_set_filter on every system), runs n_blocks 256-step warm-up blocks and
 * then times n_blocks >= 1 blocks, and writes into *best a copy of *p with the
 * fastest skin, nm_layout, list_lanes and rebuild_scope.  equil_blocks >= 0:
 * first the systems are advanced equil_blocks 256-step blocks with the default
 * parameters, and every candidate (the defaults included) starts from the
 * configuration reached, its lists built on it, so that the timing sees the list
 * lengths and the rebuild rate of a long run rather than those of the initial
 * configuration (0: every candidate starts from the given positions).  The
 * candidates change the summation order and the rebuild schedule only, not the
 * dynamics.  Pair potentials only (QTB_ERR_ARG otherwise).  stream: as qtb_init.
 * Allocates and frees one context at a time; synchronises. */
int qtb_autotune(const qtb_system *sys, int n_sys, const qtb_params *p, void *stream, int noise_mode, int n_taps,
                 double omega_max, int n_blocks, int equil_blocks, qtb_params *best, qtb_tuning *result);

/* Current step index (number of steps taken). */
int qtb_get_step(qtb_ctx *c, long long *step);

/* Cell of system sys: edges box[3] (A) and, for an isothermal-isobaric run,
 * the cell momentum p_e (eV fs; 0 otherwise).  Either pointer may be NULL.
 * Synchronises. */
int qtb_get_cell(qtb_ctx *c, int sys, double *box, double *p_e);

/* Set the cell of system sys of an isothermal-isobaric context: edges box[3]
 * (A; the initial edges times one scale lam >= 0.9, since the cell is isotropic
 * and its lists are sized for that) and cell momentum p_e (eV fs), in the form
 * qtb_get_cell reports them (after a step, before the closing half kick of the
 * cell momentum that the next step applies; whether that half kick is due is
 * left as it is).  Positions are stored relative to the cell and scale with it,
 * so a state is restored by setting the cell first and then the positions
 * (qtb_set_state takes them in the cell current at the upload).  Every list is
 * rebuilt, and the forces and the record of the current step evaluated again,
 * at the next call that needs them.  QTB_ERR_ARG for a constant-volume context,
 * an anisotropic or too small cell, or a non-finite value.  Synchronises. */
int qtb_set_cell(qtb_ctx *c, int sys, const double *box, double p_e);

/* kappa_P / (k_B T) = F_P(y), y = beta hbar w, solved in FP64 on the GPU on the
 * collocation grid y_i = y0 sinh(i t), t = asinh(y_max/y0)/(n-1), i < n:
 * least squares of Eq. 10 imposed at the nodes and midpoints with linear
 * interpolation and the asymptotic tail f(sqrt(P) y)/P + sqrt(P)/(2y) above
 * y_max.  F: [n] host output. */
int qtb_kappa_solve(int P, int n, double y_max, double y0, double *F);

/* ---- Learned kappa_P (stand-in for the solve of Eq. 10) -------------------
 * A 2-64-64-1 SiLU network maps (y = beta hbar w, P) to kappa_P/theta; inputs
 * x1 = asinh(y)/asinh(1000), x2 = (ln P - ln 2)/(ln 32 - ln 2).  It is trained on
 * the GPU (FP32 forward/backward/Adam kernels) on F_P produced by
 * qtb_kappa_solve, and the solver judges it: for each trained P the maximum
 * deviation of kappa_P/theta from the solver on held-out frequencies is kept,
 * and QTB_NOISE_QTB_PIMD_MLP uses the model only for P whose deviation is
 * within the tolerance given at training (otherwise the solver: fallback).
 * Parameters: 4417 floats, W1[64][2], b1[64], W2[64][64], b2[64], W3[64], b3.
 * The model owns its device memory (cudaMalloc); calls run on the legacy
 * default stream and synchronise. */
typedef struct qtb_kappa_model qtb_kappa_model;

/* New model with seeded uniform (He) initial weights. */
int qtb_kappa_model_create(qtb_kappa_model **out, unsigned long long seed);

/* Train on P_list (each in 2..32): n_per_P samples per P with y uniform in
 * asinh(y) on [0, asinh(1000)]; `iters` full-batch Adam steps (learning rate
 * 3e-3 decaying exponentially to 1e-5), replayed as CUDA graphs of 50 steps; tol: largest
 * accepted deviation of kappa_P/theta (e.g. 2e-3). */
int qtb_kappa_model_train(qtb_kappa_model *m, const int *P_list, int nP, int n_per_P, int iters, double tol);

/* Mean squared error loss and its gradient (4417 floats) for n samples with
 * features x[n][2] and targets t[n] (host arrays), with the current weights;
 * no update. */
int qtb_kappa_model_grad(qtb_kappa_model *m, const float *x, const float *t, int n, float *grad, float *loss);

/* Model ratio kappa_P/theta at n values of y (host arrays). */
int qtb_kappa_model_eval(qtb_kappa_model *m, int P, const double *y, int n, double *ratio);

/* Weights (4417 floats, host). */
int qtb_kappa_model_get_weights(qtb_kappa_model *m, float *w, int n);
int qtb_kappa_model_set_weights(qtb_kappa_model *m, const float *w, int n);

/* Solver-judged deviation per trained P (up to max entries), training time (ms)
 * and final loss. */
int qtb_kappa_model_info(qtb_kappa_model *m, int *P_out, double *err_out, int max, int *n_out, double *train_ms,
                         double *final_loss);

void qtb_kappa_model_destroy(qtb_kappa_model *m);

/* Use `model` (borrowed; it must outlive its use) for QTB_NOISE_QTB_PIMD_MLP. */
int qtb_set_kappa_model(qtb_ctx *c, const qtb_kappa_model *model);

/* Source of system sys's spectrum after qtb_set_filter: 0 theta (QTB) or
 * k_B T (white), 1 the kappa_P solver, 2 the learned model. */
int qtb_filter_source(qtb_ctx *c, int sys, int *source);

/* Same solve as qtb_kappa_solve for callers that cannot allocate device
 * memory (no counterpart in the paper; an interface convenience).  A process
 * whose device memory is all reserved by another allocator (a caching pool
 * that owns the device, an MPS client with a fixed memory limit) cannot get a
 * cudaMalloc through, and a latency-critical loop must not call it, since an
 * allocation can block and synchronise the device.  This entry point
 * allocates nothing: its scratch is a static __device__ array of 6.3 MB in the
 * library, present on every device that loads the library until the process
 * exits.
 *   n        collocation nodes, 8 <= n <= 512 (QTB_ERR_ARG beyond: the scratch
 *            is sized for 512)
 *   F_dev    [n] DEVICE output buffer owned by the caller (F_P at the nodes)
 *   stream   cudaStream_t to run on (NULL = legacy default stream); every call,
 *            P = 1 included, synchronises it before returning.
 * The first call on a device looks up the scratch array's device address
 * (cudaGetSymbolAddress) with that device current; make that first call before
 * any stream capture.  All calls share the one array and it keeps the last
 * call's contents (the solver clears what must start at zero): calls that
 * overlap on the GPU, from different streams or threads, race. */
int qtb_kappa_solve_noalloc(int P, int n, double y_max, double y0, double *F_dev, void *stream);

/* Measured FP32 fused-multiply-add throughput of the current GPU (TFLOP/s), the
 * denominator of the step kernel's roofline (no counterpart in the paper): every
 * SM filled with threads running independent chains of dependent FMAs, the best
 * of five timed launches of about 5 ms (*ms, may be NULL); FMA = 2 flops.  Runs on
 * the default stream and synchronises; allocates and frees 1.2 MB of device
 * memory.  QTB_ERR_ARG for a NULL tflops. */
int qtb_fp32_peak(double *tflops, double *ms);

void qtb_destroy(qtb_ctx *c);

/* Message of the last failed call in this thread (never NULL). */
const char *qtb_last_error(void);

#ifdef __cplusplus
}
#endif
#endif /* QTB_H */
