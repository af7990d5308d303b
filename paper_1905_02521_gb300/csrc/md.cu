// md.cu -- integrators, external potentials, reductions and the launchers of
// the MD hot path (sm_103a); the device code is in md_kernels.cuh.
#include "md_kernels.cuh"

namespace qtb {

// External separable potentials, one thread per bead-atom.  grid = (gx, nsys)
template <class R>
__global__ void __launch_bounds__(128) k_force_ext(Dev d, PairTabT<R> T, int kick)
{
    __shared__ double red[4][kNQ];
    const DSys S = d.sys[blockIdx.y];
    const int l = blockIdx.x * blockDim.x + threadIdx.x;
    double acc[kNQ];
#pragma unroll
    for (int q = 0; q < kNQ; ++q) acc[q] = 0.0;
    if (l < S.N * S.P) {
        const size_t G = (size_t)d.G, g = S.g0 + l;
        const int t = d.typ[g];
        const R hdtm = T.hdt_m[t];
        const R invP = sizeof(R) == 4 ? (R)S.invP_f : (R)S.invP;
        const R *X = reinterpret_cast<const R *>(d.x);
        R *Fo = reinterpret_cast<R *>(d.f);
        R *V = reinterpret_cast<R *>(d.v);
        double e = 0.0, ke = 0.0, x2 = 0.0;
        for (int c = 0; c < 3; ++c) {
            const R x = X[c * G + g];
            R fx, ex;
            if (T.potential == QTB_POT_HARMONIC) {
                const R k = T.ext_k[t];
                fx = -k * x;
                ex = R(0.5) * k * x * x;
            } else {
                const R u = x * x * T.ext_ia2 - R(1);
                fx = R(-4) * T.ext_V0 * u * x * T.ext_ia2;
                ex = T.ext_V0 * u * u;
            }
            const R fb = fx * invP;
            Fo[c * G + g] = fb;
            R v = V[c * G + g];
            if (kick) {
                v += hdtm * fb;
                V[c * G + g] = v;
            }
            e += (double)ex;
            ke += 0.5 * T.mass_mvv[t] * (double)v * (double)v;
            x2 += (double)x * (double)x;
            acc[Q_MOM + c] = T.mass[t] * (double)v;
            acc[Q_VIR + c] = (double)x * (double)fx;
        }
        acc[Q_K] = ke;
        acc[Q_V] = e;
        acc[Q_X2] = x2;
    }
    for (int q = 0; q < kNQ; ++q) acc[q] = warp_sum(acc[q]);
    cta_store_partials(acc, red, d.part + ((size_t)blockIdx.y * gridDim.x + blockIdx.x) * kNQ);}

// ---------------------------------------------------------------------------
// Per-system reduction into the observable record (external potentials).

__global__ void k_reduce(Dev d, int j, int record)
{
    __shared__ double sh[4][kNQ + 1];
    const long long step = d.clock[0] * kBlockSteps + j + 1;  // steps completed
    // during stepping only the recorded steps are reduced (record < 0: always)
    if (record >= 0 && step % d.obs_stride != 0) return;
    reduce_system(d, blockIdx.x, step, record, sh);
}

__global__ void k_tick(Dev d) { d.clock[0] += 1; }
__global__ void k_setclock(Dev d, long long b) { d.clock[0] = b; }

// ---------------------------------------------------------------------------
// launchers

bool md_supported_P(int P) { return (P >= 1 && P <= 6) || P == 8 || P == 16 || P == 32; }

int integrate_atoms_per_cta(int P, int big) { return P == 1 ? kIntAtomsPerCta : nm_atoms(P, big); }

template <int P, int PM, class R>
static void nm_launch(const Dev &d, const MdLaunch &m, int j, int cur, cudaStream_t st)
{
    if (m.nm_big) k_integrate_nm<P, PM, R, 1><<<m.n_icta, nm_threads(P, 1), nm_smem<P, PM, R>(1), st>>>(d, j, cur);
    else k_integrate_nm<P, PM, R, 0><<<m.n_icta, nm_threads(P, 0), nm_smem<P, PM, R>(0), st>>>(d, j, cur);
}

template <int P, int PM, class R>
static cudaError_t nm_prepare_one(int big)
{
    if (big) return cudaFuncSetAttribute(k_integrate_nm<P, PM, R, 1>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)nm_smem<P, PM, R>(1));
    return cudaFuncSetAttribute(k_integrate_nm<P, PM, R, 0>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)nm_smem<P, PM, R>(0));
}

template <int PM, class R>
static cudaError_t nm_prepare(const MdLaunch &m)
{
    for (int u = 0; u < m.nP; ++u) {
        cudaError_t e = cudaSuccess;
        switch (m.Pvals[u]) {
#define QTB_P(PP) case PP: e = nm_prepare_one<PP, PM, R>(m.nm_big); break;
            QTB_P(2) QTB_P(3) QTB_P(4) QTB_P(5) QTB_P(6) QTB_P(8) QTB_P(16) QTB_P(32)
#undef QTB_P
            default: break;
        }
        if (e != cudaSuccess) return e;
    }
    return cudaSuccess;
}

cudaError_t integrate_prepare(const MdLaunch &m)
{
    if (!m.pair) return m.mixed ? nm_prepare<PM_FREE, float>(m) : nm_prepare<PM_FREE, double>(m);
    return m.mixed ? nm_prepare<PM_FIX, float>(m) : nm_prepare<PM_BOX64, double>(m);
}

template <int PM, class R>
static void integrate_all(const Dev &d, const MdLaunch &m, int j, int cur, cudaStream_t st)
{
    for (int u = 0; u < m.nP; ++u) {
        switch (m.Pvals[u]) {
            case 1: k_integrate<1, PM, R><<<m.n_icta, 128, 0, st>>>(d, j, cur); break;
#define QTB_P(PP) case PP: nm_launch<PP, PM, R>(d, m, j, cur, st); break;
            QTB_P(2) QTB_P(3) QTB_P(4) QTB_P(5) QTB_P(6) QTB_P(8) QTB_P(16) QTB_P(32)
#undef QTB_P
            default: break;
        }
    }
}

void launch_integrate(const Dev &d, const MdLaunch &m, int j, int cur, cudaStream_t st)
{
    if (!m.pair) {
        if (m.mixed) integrate_all<PM_FREE, float>(d, m, j, cur, st);
        else integrate_all<PM_FREE, double>(d, m, j, cur, st);
    } else {
        if (m.mixed) integrate_all<PM_FIX, float>(d, m, j, cur, st);
        else integrate_all<PM_BOX64, double>(d, m, j, cur, st);
    }
}

cudaError_t step_prepare(MdLaunch &m, int stage_entries)
{
    if (m.lanes == 8) return step_prepare_l8(m, stage_entries);
    if (m.lanes == 32) return step_prepare_l32(m, stage_entries);
    return step_prepare_l16(m, stage_entries);
}

cudaError_t launch_force(const Dev &d, const MdLaunch &m, const PairTabT<float> &Tf, const PairTabT<double> &Td,
                         int kick, int j, int cur, int adv, int rec, cudaStream_t st)
{
    if (m.pair) {
        if (m.lanes == 8) return step_force_l8(d, m, Tf, Td, kick, j, cur, adv, rec, st);
        if (m.lanes == 32) return step_force_l32(d, m, Tf, Td, kick, j, cur, adv, rec, st);
        return step_force_l16(d, m, Tf, Td, kick, j, cur, adv, rec, st);
    }
    dim3 g((unsigned)m.n_ecta, (unsigned)d.nsys);
    if (m.mixed) k_force_ext<float><<<g, 128, 0, st>>>(d, Tf, kick);
    else k_force_ext<double><<<g, 128, 0, st>>>(d, Td, kick);
    return cudaGetLastError();
}

void launch_reduce(const Dev &d, const MdLaunch &m, int j, int record, cudaStream_t st)
{
    k_reduce<<<d.nsys, 128, 0, st>>>(d, j, record);
}

void launch_tick(const Dev &d, cudaStream_t st) { k_tick<<<1, 1, 0, st>>>(d); }
void launch_setclock(const Dev &d, long long b, cudaStream_t st) { k_setclock<<<1, 1, 0, st>>>(d, b); }

}  // namespace qtb
