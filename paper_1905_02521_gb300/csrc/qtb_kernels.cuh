// qtb_kernels.cuh -- launcher declarations shared by the host code and the
// CUDA translation units.
#pragma once
#include "qtb_dev.cuh"

namespace qtb {

enum { FK_FP64 = 0, FK_FP32 = 1, FK_BF16 = 2 };  // filter / ring arithmetic

// Spectrum parameters of one system (set_filter).
struct DSpec {
    int mode, K, taps0, P;
    double dt, T, omega_max;
    const double *F;  // kappa_P grid (device) for QTB-PIMD
    int n;
    double ymax, y0;
};

// capi.cu: record the message returned by qtb_last_error(); returns code
int set_last_error(int code, const char *msg);

// mlp.cu: learned kappa_P model (device weights, solver-judged acceptance per P)
const float *kappa_model_weights(const qtb_kappa_model *M);
bool kappa_model_accepts(const qtb_kappa_model *M, int P);

// noise.cu
void launch_white(const Dev &d, int filter_kind, int max_dofp, int nsys, long long blk, cudaStream_t st);
void launch_filter_simt(const Dev &d, int filter_kind, int max_dofp, int nsys, int Kmax, cudaStream_t st);
cudaError_t filter_simt_prepare(int Kmax);
void launch_spectrum_taps(const DSpec *spec, int nsys, int Kmax, double *S, double *h64, float *h32,
                          const float *mlp_w, cudaStream_t st);

// mlp.cu: spectrum S_j = kT f(y_j) ratio_model(y_j, P) W(w_j) for systems in the learned mode
void launch_spectrum_mlp(const DSpec *spec, int nsys, int Kmax, double *S, const float *w, cudaStream_t st);
// Fourier-segment generator (Eq. 9), segments of n = 256 M <= 2048 steps:
// sqrt(S_j / n) per system on the segment grid, then the segment of every dof
// into eta rows 0..n-1 (only at a segment's first block unless force)
size_t fourier_smem(int n, int fp64);
cudaError_t fourier_prepare(int n);
void launch_spectrum_seg(const DSpec *spec, int nsys, int n, void *sq, int fp64, cudaStream_t st);
void launch_fourier(const Dev &d, int fp64, int max_dofp, int nsys, const void *sq, const void *tw, int n, int force,
                    cudaStream_t st);
// kappa_P solve on the collocation grid (Eq. 10): A [(2n-1) x n], b [2n-1], M [n x n]
// scratch, work [(2n-1) + n] scratch of the refinement steps, r [n] the solution
constexpr int kKappaRefine = 1;  // corrected semi-normal-equation refinement steps
void launch_kappa_solve(int P, int n, double ymax, double y0, double *A, double *b, double *M, double *r,
                        double *work, unsigned *err, cudaStream_t st);

// md.cu
struct MdLaunch {
    int mixed;            // 0: FP64 form, 1: mixed form
    int pair;             // pair potential (else external)
    int n_icta;           // integrator CTAs
    int n_ccta;           // centroid-estimator CTAs (0: no ring polymer)
    int n_ecta;           // external-force CTAs per system
    int nP;               // number of distinct bead counts
    int Pvals[8];         // distinct bead counts
    int fused;            // all systems one-bead with a pair potential: the step kernel
                          // carries out the first half of the next step
    int nm_big;           // ring-polymer integrator with 32 atoms per CTA (large contexts)
    int lanes;            // lanes per bead-atom of the step kernel (8, 16, 32)
    int step_grid[4];     // resident CTAs of the step kernel, by (adv, rec)
    int minimg;           // mixed form, fixed cells all larger than 2 (r_cut + 2 skin): the step
                          // kernel variant that takes list displacements by minimum image
    size_t step_smem;     // its dynamic shared memory (list build staging chunk)
};
constexpr int kIntAtomsPerWarp = 10;                   // integrator: lanes 3a + c, a < 10
constexpr int kIntAtomsPerCta = 4 * kIntAtomsPerWarp;  // 128 threads
constexpr int kStencilCells = 125;                     // 5^3 stencil of (r_cut + skin)/2 cells
// attributes and resident grid sizes of the cooperative step kernel (m.lanes)
cudaError_t step_prepare(MdLaunch &m, int stage_entries);
// per lane count, one translation unit each (md_step8.cu, md_step16.cu, md_step32.cu)
cudaError_t step_prepare_l8(MdLaunch &m, int stage_entries);
cudaError_t step_prepare_l16(MdLaunch &m, int stage_entries);
cudaError_t step_prepare_l32(MdLaunch &m, int stage_entries);
cudaError_t step_force_l8(const Dev &d, const MdLaunch &m, const PairTabT<float> &Tf, const PairTabT<double> &Td,
                          int kick, int j, int cur, int adv, int rec, cudaStream_t st);
cudaError_t step_force_l16(const Dev &d, const MdLaunch &m, const PairTabT<float> &Tf, const PairTabT<double> &Td,
                           int kick, int j, int cur, int adv, int rec, cudaStream_t st);
cudaError_t step_force_l32(const Dev &d, const MdLaunch &m, const PairTabT<float> &Tf, const PairTabT<double> &Td,
                           int kick, int j, int cur, int adv, int rec, cudaStream_t st);
// positions of step s: the integrator writes pos[cur], cur = s & 1, and
// requests a list rebuild in flag[cur] when some bead-atom moved skin/2
void launch_integrate(const Dev &d, const MdLaunch &m, int j, int cur, cudaStream_t st);
// one step's force (pair potential: the cooperative step kernel, which first
// rebuilds the lists when flag[cur] is set).  kick: closing B step; adv: also
// the first half of step j + 1, positions to pos[cur ^ 1]; rec: the step may
// be recorded, then the kernel also reduces the observables
cudaError_t launch_force(const Dev &d, const MdLaunch &m, const PairTabT<float> &Tf, const PairTabT<double> &Td,
                         int kick, int j, int cur, int adv, int rec, cudaStream_t st);
void launch_reduce(const Dev &d, const MdLaunch &m, int j, int record, cudaStream_t st);
// centroid-virial estimators of the ring-polymer systems (record slots 18, 19),
// after the force launch of a step that may be recorded (record < 0: latest only)
constexpr int kCenAtoms = 32;  // atoms per CTA of the centroid estimator
void launch_centroid(const Dev &d, const MdLaunch &m, int j, int record, int kick, cudaStream_t st);
// spring energy of the current positions into the integrator partials (the
// record of a refreshed step, which no integrator produced)
void launch_spring(const Dev &d, const MdLaunch &m, cudaStream_t st);
// positions / velocities (either may be null) of system s, [P][N][3] FP64 in device
// memory (n3 = 3 N P values), into the state (wrapped / fixed point as the form needs;
// near_ref, pair potentials with lists built: each position as its periodic copy
// nearest the reference position of the last rebuild)
void launch_load_state(const Dev &d, const MdLaunch &m, int s, long long n3, const double *pos, const double *vel,
                       int near_ref, cudaStream_t st);
// positions (which 0, wrapped for pair potentials), velocities (1) or forces (2) of
// system s into out[P][N][3] (FP64, device memory, n3 = 3 N P values)
void launch_store_state(const Dev &d, const MdLaunch &m, int s, long long n3, int which, double *out, cudaStream_t st);
// pair potentials, before the forces of an uploaded state: packed positions of
// every bead-atom into pos[cur]; rebuild requests (flag, rflag[cur]) for the
// systems with a bead-atom more than skin/2 from its position at the last rebuild
void launch_refresh_check(const Dev &d, const MdLaunch &m, int cur, cudaStream_t st);
// isothermal-isobaric cells: update at the start of step j (see md.cu)
void launch_cell(const Dev &d, int j, bool fp32, cudaStream_t st);
int measure_fp32_peak(double *tflops, double *ms);  // peak.cu
// words[0]: a flag nothing sets; words[1]: set to 1 when the bounded wait gives up
void launch_wait_selftest(unsigned *words, cudaStream_t st);
void launch_tick(const Dev &d, cudaStream_t st);
void launch_setclock(const Dev &d, long long blk, cudaStream_t st);
bool md_supported_P(int P);
// atoms per CTA of the integrator for bead count P (big: large-context layout)
int integrate_atoms_per_cta(int P, int big);
// dynamic shared memory attributes of the ring-polymer integrator
cudaError_t integrate_prepare(const MdLaunch &m);

// filter_tc.cu
cudaError_t filter_tc_prepare();
void launch_build_toeplitz(const Dev &d, void *Bt, int Ktot, int Ke, cudaStream_t st);
void launch_filter_tc(const Dev &d, const void *tmapA, const void *tmapB, int n_mtiles, const int *mtile_sys,
                      cudaStream_t st);

}  // namespace qtb
