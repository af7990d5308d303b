// qtb_dev.cuh -- device-side definitions shared by the CUDA translation units
// of the QTB / QTB-PIMD hot path (sm_103a).
//
// Method: Dammak, Hayoun, Brieuc, Geneste, "Nuclear quantum effects in
// molecular dynamics simulations" (Eqs. 1, 3-5, 6-8, 10-12).
#pragma once
#include <cuda_runtime.h>
#include <stdint.h>

#include "../../include/qtb.h"

namespace qtb {

// Physical constants (CODATA 2018) and unit conversions: A, fs, eV, u, e, K.
constexpr double kHbar = 0.6582119569;          // eV fs
constexpr double kBoltz = 8.617333262e-5;       // eV / K
constexpr double kMvv2e = 103.64269652680505;   // eV per u A^2 / fs^2
constexpr double kCoulomb = 14.3996454784;      // e^2 / (4 pi eps0), eV A
constexpr double kPi = 3.14159265358979323846;

constexpr int kBlockSteps = 256;     // noise block length (steps)
constexpr int kDofPad = 128;         // per-system dof padding (tensor-core M tile)
constexpr int kNQ = 16;              // partial sums per CTA (see Q_* below)
constexpr int kRedGroup = 16;        // force units per group of the two-level record reduction
constexpr int kFixBits = 30;         // fixed-point positions: box edge = 2^30 units
constexpr int kMaxTypes = 4;
constexpr int kWarpsPerForceCta = 8;  // warps of the list build kernel

// partial-sum slots
enum { Q_K = 0, Q_V = 1, Q_SPRING = 2, Q_VIR = 3 /* 6 slots: xx yy zz xy xz yz */, Q_MOM = 9 /* 3 */,
       Q_X2 = 12 };

// position storage modes
enum { PM_BOX64 = 0, PM_FIX = 1, PM_FREE = 2 };

// device error word bits
enum { ERR_OVERFLOW = 1, ERR_NONFINITE = 2, ERR_SOLVE = 4, ERR_TIMEOUT_TC = 8, ERR_NBR_OVERFLOW = 16, ERR_TIMEOUT_BAR = 32,
       ERR_CELL = 64 };

// Isothermal-isobaric cell (isotropic Langevin barostat) of one system.  The
// stored positions stay in the reference cell (edges DSys::box, fixed point per
// reference edge in the mixed form); physical positions are lam times them, so a
// change of the cell rescales every distance without touching the state.  The
// cell kernel updates the cell at the start of each step and leaves there the
// step's coefficients for the integrator and the step kernel.
constexpr double kCellMinScale = 0.9;  // smallest lam the cell lists are sized for
// Isothermal-isobaric runs split the list skin between the cell and the
// particles: a rebuild when lam has moved by more than tol lam_rb since the last
// rebuild (tol = kNptCellSkin skin / r_list) or a bead-atom by more than D
// (physical).  A pair within r_cut now was within (lam_rb/lam) r_cut + 2 lam_rb d
// <= (r_cut tol + 2 D)/(1 - tol) of each other at the rebuild, which D = (skin
// (1 - tol) - tol r_cut)/2 makes r_cut + skin: the lists hold it.  The cell's
// volume fluctuates by a few tenths of a percent in lam, so an eighth of the skin
// (over the list radius) leaves most of the skin to the particles.
constexpr double kNptCellSkin = 0.125;
struct DNpt {
    double lam, lam_rb, peps;  // cell scale, its value at the system's last list rebuild, cell momentum (eV fs)
    double W, pext, ce, sige, alpha, V0;  // mass, P_ext, exp(-gamma_e dt), sqrt((1 - ce^2) W kT), 1 + 3/N_f, V at lam 1
    // this step: first B  v <- v e1 + (hdt/m) F g1;  A  x_ref += v a1, then v' a2;
    // closing B  v <- v e2 + (hdt/m) F g2
    double e1, g1, a1, a2, e2, g2;
    float e1f, g1f, a1f, a2f, e2f, g2f, lamf, inv_wf;  // the FP32 form's coefficients, 1/W
    int on, pending;  // barostat on; the previous step's closing half kick of the cell is due
    int pad2[2];
    double rb_tol;    // list rebuild when |lam - lam_rb| > rb_tol lam_rb (kNptCellSkin skin over the list radius)
    double lam_old, inv_lam;  // this step's lam before the update and 1/lam after (ring polymers)
    float lam_oldf, inv_lamf;
};

// Neighbour-list entry (32 bits): replica-local index j in bits 0..25, the
// periodic image m of the entry (per component m mod 4, two bits each: x at
// bit 26, y at 28, z at 30).  With 30-bit fixed point the image shift is
// (m mod 4) * 2^30, exact in wrapping 32-bit arithmetic.
constexpr unsigned kNbIdx = (1u << 26) - 1u;
constexpr int kMaxCellCap = 512;        // slots per cell of the cell list
constexpr int kListWarps = 4;        // warps per CTA of the list force kernel
// lanes per home bead-atom of the step kernel: 8, 16 (default) or 32; a force
// unit (one CTA's share of work) holds list_atoms(lanes) bead-atoms
__host__ __device__ constexpr int list_atoms(int lanes) { return kListWarps * 32 / lanes; }

struct DSys {
    int N, P;          // atoms, beads
    int g0;            // first bead-atom index (bead-major: g = g0 + b N + i)
    int dof0;          // first noise dof (dof = dof0 + (k*3 + c) N + i)
    int dofp;          // padded dof count of this system (multiple of kDofPad)
    int K;             // filter half length (taps h_0..h_K)
    int taps0;         // offset of h_0 in the taps arrays
    int rep0;          // first replica (pair potential)
    int icta0, icta1;  // integrator CTA range
    int fcta0, fcta1;  // force CTA range
    int grp0, ngrp;    // its groups of kRedGroup force units (two-level record reduction)
    int ccta0, ccta1;  // centroid-estimator CTA range (empty for one bead)
    int cell0, cell1;  // cells of all its replicas (pair potential)
    int rot0;          // offset of this system's mode rotation table
    int nm0;           // offset of this system's normal-mode matrix
    double box[3];
    double T, gamma, c1, wP;
    float fix_scale[3];      // box / 2^30 (A per fixed-point unit)
    float fix_inv[3];        // 2^30 / box
    float invP_f, c1_f;      // 1/P, c1 in FP32
    double invP;
    // neighbour-list validity: a bead-atom may move (skin/2) since the last
    // rebuild; squared, in A^2
    double skin2;
    float skin2_f;
    // its list radius (r_cut + its skin), squared
    double rl2;
    float rl2_f;
    // isothermal-isobaric cells: the physical displacement D allowed since the
    // last rebuild, squared (A^2), D = (skin (1 - tol) - tol r_cut)/2 with the
    // cell's share tol = kNptCellSkin skin / (r_cut + skin) of the list radius
    double npt_d2;
    float npt_d2_f;
};

struct DRep {          // one replica (system, bead) of a pair-potential system
    int sys, g0, N;
    int nc[3];         // cells per edge
    int cell0;         // first cell
    int cta0;          // first binning CTA
    int fcta0;         // first force unit of the step kernel
    double box[3];
    float fix_scale[3];  // box / 2^30
};

// Interaction table in the arithmetic type R of the force kernel (no FP64
// arithmetic leaks into the FP32 kernels).  Index of a type pair: a * kMaxTypes + b.
template <class R> struct PairTabT {
    R A[kMaxTypes * kMaxTypes], inv_rho[kMaxTypes * kMaxTypes], A_over_rho[kMaxTypes * kMaxTypes];
    R C[kMaxTypes * kMaxTypes], C6[kMaxTypes * kMaxTypes];
    R qq[kMaxTypes * kMaxTypes];      // k_e q_a q_b
    R eshift[kMaxTypes * kMaxTypes];  // Buckingham energy at r_cut
    R alpha, alpha2, two_a_sqrtpi, rc, rc2, erfc_rc_over_rc, fshift;  // DSF constants
    // FP32 form only: exp(-alpha^2 r^2) = 2^(-r^2 alpha^2 log2 e); erfc(x) =
    // exp(-x^2) P(u), u = x us - 1 in [-1, 1] on 0 <= x <= alpha r_cut, P a
    // degree-11 Chebyshev interpolant of exp(x^2) erfc(x) made at context
    // creation (relative error ~2e-7 in FP32)
    R alpha2_l2e, erfc_us;
    R rl2;                            // (r_cut + skin)^2: neighbour-list radius
    R erfc_c[12];
    R hdt_m[kMaxTypes];               // dt / (2 m mvv2e)
    R ext_k[kMaxTypes];               // HARMONIC: m mvv2e w0^2
    R ext_V0, ext_ia2;                // DOUBLEWELL: V0, 1/a^2
    double mass[kMaxTypes];           // u (momentum)
    double mass_mvv[kMaxTypes];       // m mvv2e (kinetic energy, FP64 accumulation)
    float2 mass_ff[kMaxTypes], half_mvv_ff[kMaxTypes];  // m, m mvv2e / 2 as float-float (hi, lo)
    int ntypes, potential;
};
typedef PairTabT<double> PairTab;

// Everything a kernel needs, passed by value.
struct Dev {
    // sizes
    int nsys, nrep, ncells, cap;
    long long G;                      // bead-atoms
    long long Dtot;                   // padded dofs
    int Kb, nslots;                   // noise ring: blocks of half-span, slots
    int obs_stride, max_records;
    double dt;
    // tables
    const DSys *sys;
    const DRep *rep;
    const int *cell_rep;  // [ncells]
    const int *lcta_rep;  // [nunits] replica of each force unit
    int nunits;           // force units
    const int *icta_sys;  // [integrator CTAs] system of each CTA
    const int *ext_cta_sys;
    // state
    void *x;              // positions, SoA [3][G] (double, int32 or R by mode)
    void *v;              // velocities [3][G] (R)
    void *f;              // forces [3][G] (R), already multiplied by 1/P
    const int *typ;       // [G] type of each bead-atom
    // cells
    int *cnt;             // [ncells] running counts (binning)
    int *ccount;          // [ncells] counts after sorting
    int *cidx;            // [ncells * cap] bead-atom index, sorted
    void *cpos;           // [ncells * cap] packed {x, y, z, replica-local index} (int4 or 4 doubles)
    // neighbour lists (pair potential)
    void *pos[2];         // [G] packed {x, y, z, type} (int4 or 4 doubles); step s reads pos[s & 1]
    void *xref;           // [3][G] positions at the last rebuild (type of x)
    unsigned *nbr;        // [G][maxnb] list entries (see kNbIdx)
    int *nnb;             // [G] entries per bead-atom
    int maxnb;
    unsigned *flag;       // [2] rebuild requests; flag[s & 1] is set by whoever produces the positions of step s
    unsigned *rflag;      // [2][nsys] the same per system: a rebuild covers the requesting systems
    int rebuild_all;      // ... or every system (rebuild scope 1)
    unsigned *gbar;       // [2] grid barrier of the cooperative step kernel: arrivals, generation
    unsigned long long *nrebuild;  // list rebuilds carried out
    int eta_blocks;       // blocks per noise segment (1: time-domain filter)
    // noise
    void *ring;           // [nslots][Dtot][256] white noise (double, float or bf16)
    void *eta;            // [256][Dtot] coloured noise (R)
    const double *taps64; // FP64 taps
    const void *tapsR;    // taps in the filter type
    // integrator tables
    const void *rot;      // [sum P][3] (cos, sin/w, -w sin) per mode (R)
    const void *nmC;      // normal-mode matrices (R)
    const void *hdt_m;    // [ntypes] dt / (2 m mvv2e) (R)
    const void *osig;     // [nsys * ntypes] sqrt((1 - c1^2)/(m mvv2e)) (R)
    // reductions
    double *part;         // [CTAs][kNQ] (the FP32 list kernel: float-float pairs)
    double *gpart;        // [groups][kNQ] sums of kRedGroup units' partials (list kernel)
    unsigned *gdone;      // [groups] units finished, reset by the group's last one
    double *ipart;        // [integrator CTAs][kNQ]
    DNpt *npt;            // [nsys] isothermal-isobaric cells (null: constant volume)
    double *latest;       // [nsys][QTB_NREC]
    double *series;       // [max_records][nsys][QTB_NREC]
    long long *clock;     // [0] = current noise block
    unsigned *err;        // error word
    unsigned *done;       // [nsys] CTAs finished (last-CTA reduction), reset by the last one
    double *cpart;        // [centroid CTAs][kCenQ] virial term, K_0, the cell kick's dK and momentum
    const int *ccta_sys;  // [centroid CTAs] system of each CTA
    unsigned *cdone;      // [nsys] centroid CTAs finished, reset by the last one
    int stage_cap;        // staged neighbourhood entries per CTA of the list build kernel
    unsigned long long seed;
    double mass_mvv[kMaxTypes];  // m * mvv2e per type (eV fs^2 / A^2)
};

// -------------------------------------------------------------------------
// Philox4x32-10 (Salmon et al., SC'11), written from its published
// definition; counter = (lo32(q), dof, stream, hi32(q)), q = floor(n/4),
// key = (lo32(seed), hi32(seed) ^ sys).
__device__ __forceinline__ uint4 philox4x32_10(uint4 c, uint32_t k0, uint32_t k1)
{
#pragma unroll
    for (int r = 0; r < 10; ++r) {
        if (r > 0) { k0 += 0x9E3779B9u; k1 += 0xBB67AE85u; }
        uint32_t hi0 = __umulhi(0xD2511F53u, c.x), lo0 = 0xD2511F53u * c.x;
        uint32_t hi1 = __umulhi(0xCD9E8D57u, c.z), lo1 = 0xCD9E8D57u * c.z;
        c = make_uint4(hi1 ^ c.y ^ k0, lo1, hi0 ^ c.w ^ k1, lo0);
    }
    return c;
}

__host__ __device__ inline long long floor_div(long long a, long long b)
{
    long long q = a / b;
    return (q * b > a) ? q - 1 : q;
}

// sign-extend a 30-bit fixed-point difference (minimum image)
__device__ __forceinline__ int fix_minimg(int d) { return (d << (32 - kFixBits)) >> (32 - kFixBits); }

// row of the coloured-noise buffer for step j of the current block: the
// Fourier-segment generator keeps segments of eta_blocks blocks (256 rows each)
__device__ __forceinline__ size_t eta_row(const Dev &d, int j)
{
    if (d.eta_blocks <= 1) return (size_t)j;
    const long long b = d.clock[0];
    return (size_t)(b - floor_div(b, d.eta_blocks) * d.eta_blocks) * kBlockSteps + j;
}

}  // namespace qtb
