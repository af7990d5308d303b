// md.cu -- the launchers of the MD hot path (sm_103a) and its smaller kernels:
// external potentials, reductions, centroid-virial estimators, the spring term
// of refreshed records, state upload and download, the bounded-wait self-test.
// The step kernel and the integrators are in md_kernels.cuh and md_integrate.cuh.
#include "md_integrate.cuh"

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
    reduce_system<false>(d, blockIdx.x, step, record, sh, d.part, d.sys[blockIdx.x].fcta0, d.sys[blockIdx.x].fcta1);
}

// ---------------------------------------------------------------------------
// Centroid-virial kinetic estimators of the ring-polymer systems (P > 1), on
// the recorded steps, after the force kernel (positions and forces of the step,
// velocities after the closing kick):
//   slot 18: K_cv   = 3N k_B T/2 - 1/2 sum_i sum_s (r_i,s - rbar_i) . f_i,s
//   slot 19: K_cv,0 = K_0        - 1/2 sum_i sum_s (r_i,s - rbar_i) . f_i,s,
// f = -(1/P) grad V (Eq. 4), rbar the atom's bead centroid, K_0 = sum_i m_i P
// |vbar_i|^2 / 2 the kinetic energy of the centroid mode (the form for a bath
// that does not hold the centroid at k_B T, QTB-PIMD).  A CTA takes kCenAtoms
// atoms (lane = atom, coalesced rows); its 8 warps split the beads.  Per atom and
// component, with d_b the offset of bead b from bead 0 (minimum image), two
// passes over the beads give dbar, then sum_b (d_b - dbar) f_b, in the
// arithmetic of the form (FP32 form: sums over atoms in float-float; the FP64
// pipe of this GPU is slow).  The last CTA of a system completes the record
// (fixed order, FP64); slots 21
// and 22 are K_0 and the centroid virial (1/P) sum_s W_s - sum (r - rbar) . f.
// In an isothermal-isobaric cell (every step, kick = 1) this kernel also ends
// the step's closing B(dt/2) of each centroid with the cell's friction (the
// force kernel gave the plain kick) and adds the change to the record's K,
// E_prim and momentum; bead offsets are physical (lam times the stored ones).
constexpr int kCenWarps = 8;
constexpr int kCenQ = 6;  // per-CTA partials: virial term, K_0, and the cell kick's dK and momentum

template <int PM, class R>
__global__ void __launch_bounds__(32 * kCenWarps) k_centroid(Dev d, int j, int record, int kick)
{
    typedef typename PosT<PM, R>::S PS;
    constexpr bool kF32 = sizeof(R) == 4;
    constexpr int NB = (32 + kCenWarps - 1) / kCenWarps;  // beads per warp (P <= 32)
    __shared__ R sh[kCenWarps][9][kCenAtoms];
    __shared__ R scv[kCenWarps][kCenAtoms];
    __shared__ double fin[kCenWarps][kCenQ];
    __shared__ int last;
    const long long step = d.clock[0] * kBlockSteps + j + 1;  // steps completed
    // (isothermal-isobaric cells need K_0 and W_cv on every step)
    if (record >= 0 && step % d.obs_stride != 0 && !d.npt) return;
    const int cta = blockIdx.x, s = d.ccta_sys[cta];
    const DSys S = d.sys[s];
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int N = S.N, P = S.P;
    const int i = (cta - S.ccta0) * kCenAtoms + lane;
    const size_t G = (size_t)d.G;
    const PS *X = reinterpret_cast<const PS *>(d.x);
    const R *F = reinterpret_cast<const R *>(d.f);
    R *V = reinterpret_cast<R *>(d.v);
    // stored positions are the physical ones over lam in a cell
    const DNpt *NC = (d.npt && d.npt[s].on) ? d.npt + s : nullptr;
    const R lam = NC ? (kF32 ? (R)NC->lamf : (R)NC->lam) : R(1);
    const R invP = kF32 ? (R)S.invP_f : (R)S.invP;
    const bool cellkick = NC && kick;
    // pass 1: this warp's beads (b = warp, warp + 8, ...): offsets from bead 0,
    // forces, and their sums with the velocities'
    R dv[3][NB], fv[3][NB], sd[3], sf[3], sv[3];
#pragma unroll
    for (int c = 0; c < 3; ++c) {
        sd[c] = sf[c] = sv[c] = R(0);
#pragma unroll
        for (int k = 0; k < NB; ++k) dv[c][k] = fv[c][k] = R(0);
        if (i < N) {
            const size_t o0 = (size_t)c * G + S.g0 + i;
            const PS x0 = X[o0];
#pragma unroll
            for (int k = 0; k < NB; ++k) {
                const int b = warp + k * kCenWarps;
                if (b < P) {
                    const size_t o = o0 + (size_t)b * N;
                    const R dd = PosT<PM, R>::rel(X[o], x0, S.box[c], S.fix_scale[c], S.fix_inv[c]) * lam;
                    const R f = F[o];
                    dv[c][k] = dd;
                    fv[c][k] = f;
                    sd[c] += dd;
                    sf[c] += f;
                    sv[c] += V[o];
                }
            }
        }
        sh[warp][c][lane] = sd[c];
        sh[warp][3 + c][lane] = sf[c];
        sh[warp][6 + c][lane] = sv[c];
    }
    __syncthreads();
    // the atom's bead sums (every warp forms them alike, in warp order)
#pragma unroll
    for (int c = 0; c < 3; ++c) {
        sd[c] = sf[c] = sv[c] = R(0);
        for (int w = 0; w < kCenWarps; ++w) {
            sd[c] += sh[w][c][lane];
            sf[c] += sh[w][3 + c][lane];
            sv[c] += sh[w][6 + c][lane];
        }
    }
    // pass 2: the virial term sum_b (d_b - dbar) . f_b over this warp's beads and,
    // in a cell, the closing B(dt/2) of the centroid with the cell's friction: the
    // force kernel gave every bead the plain kick hdt f / m; the centroid velocity
    // becomes vbar e2 + (hdt/m) fbar g2 (vbar before the kick)
    R cvw = R(0), del[3] = {R(0), R(0), R(0)};
    int ty = 0;
    if (i < N) {
        ty = d.typ[S.g0 + i];
        R e2 = R(1), g2 = R(1), hd = R(0);
        if (cellkick) {
            e2 = kF32 ? (R)NC->e2f : (R)NC->e2;
            g2 = kF32 ? (R)NC->g2f : (R)NC->g2;
            hd = reinterpret_cast<const R *>(d.hdt_m)[ty];
        }
#pragma unroll
        for (int c = 0; c < 3; ++c) {
            const R dbar = sd[c] * invP;
#pragma unroll
            for (int k = 0; k < NB; ++k)
                if (warp + k * kCenWarps < P) cvw = fma(dv[c][k] - dbar, fv[c][k], cvw);
            if (cellkick) {
                const R vb = sv[c] * invP, fb = hd * (sf[c] * invP);
                del[c] = fma(vb - fb, e2, fb * g2) - vb;
                const size_t o0 = (size_t)c * G + S.g0 + i;
#pragma unroll
                for (int k = 0; k < NB; ++k) {
                    const int b = warp + k * kCenWarps;
                    if (b < P) V[o0 + (size_t)b * N] += del[c];
                }
            }
        }
    }
    scv[warp][lane] = cvw;
    __syncthreads();
    if (warp == 0) {
        // per atom: the virial term, K_0 after the kick, and the kick's change of K
        // and of the momentum; then the sums over the CTA's atoms (FP32 form in
        // float-float, FP64 form in FP64)
        R q[kCenQ];
#pragma unroll
        for (int u = 0; u < kCenQ; ++u) q[u] = R(0);
        if (i < N) {
            for (int w = 0; w < kCenWarps; ++w) q[0] += scv[w][lane];
            const double mv = d.mass_mvv[ty];
            const R hmP = (R)(0.5 * mv * P), mP = (R)(mv * (1.0 / kMvv2e) * P);
            R k0 = R(0), dk = R(0);
#pragma unroll
            for (int c = 0; c < 3; ++c) {
                const R vb = sv[c] * invP, vn = vb + del[c];
                k0 = fma(vn, vn, k0);
                dk = fma(del[c], vn + vb, dk);
                q[3 + c] = mP * del[c];
            }
            q[1] = hmP * k0;
            q[2] = hmP * dk;
        }
        double out[kCenQ];
#pragma unroll
        for (int u = 0; u < kCenQ; ++u) {
            if constexpr (kF32) {
                FF a{(float)q[u], 0.f};
                a.warp_reduce();
                out[u] = (double)a.hi + (double)a.lo;
            } else {
                out[u] = warp_sum((double)q[u]);
            }
        }
        if (lane == 0)
            for (int u = 0; u < kCenQ; ++u) d.cpart[kCenQ * (size_t)cta + u] = out[u];
    }
    // the CTA that finishes a system last completes its record
    __threadfence();
    __syncthreads();
    if (threadIdx.x == 0) last = (atomicAdd(&d.cdone[s], 1u) == (unsigned)(S.ccta1 - S.ccta0 - 1)) ? 1 : 0;
    __syncthreads();
    if (!last) return;
    __threadfence();
    double t[kCenQ];
#pragma unroll
    for (int u = 0; u < kCenQ; ++u) t[u] = 0.0;
    for (int c = S.ccta0 + (int)threadIdx.x; c < S.ccta1; c += blockDim.x)
#pragma unroll
        for (int u = 0; u < kCenQ; ++u) t[u] += __ldcg(d.cpart + kCenQ * (size_t)c + u);
#pragma unroll
    for (int u = 0; u < kCenQ; ++u) {
        t[u] = warp_sum(t[u]);
        if (lane == 0) fin[warp][u] = t[u];
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        double tot[kCenQ];
        for (int u = 0; u < kCenQ; ++u) {
            tot[u] = 0.0;
            for (int w = 0; w < kCenWarps; ++w) tot[u] += fin[w][u];
        }
        const double cv = tot[0], k0 = tot[1];
        double *L = d.latest + (size_t)s * QTB_NREC;
        if (cellkick) {  // the record of the force kernel had the plain kick
            L[1] += tot[2];
            L[4] += tot[2];
            for (int c = 0; c < 3; ++c) L[14 + c] += tot[3 + c];
        }
        L[18] = 1.5 * N * kBoltz * S.T - 0.5 * cv;
        L[19] = k0 - 0.5 * cv;
        L[21] = k0;
        L[22] = (L[5] + L[9]) + L[13] - cv;
        if (record >= 0 && step % d.obs_stride == 0) {
            const long long r = step / d.obs_stride - 1;
            const int slot = (int)(r % d.max_records);
            double *Sr = d.series + ((size_t)slot * d.nsys + s) * QTB_NREC;
            const int upd[9] = {1, 4, 14, 15, 16, 18, 19, 21, 22};
            for (int u = 0; u < 9; ++u) Sr[upd[u]] = L[upd[u]];
        }
        d.cdone[s] = 0u;
    }
}

// Spring energy of the current positions into the integrator partials, for the
// record of a step that no integrator produced (forces refreshed after qtb_init
// or qtb_set_state; the partials would otherwise be stale or unset).  The CTAs
// of the integrator grid split each system's atoms evenly; the sum over a
// system's partials is what the reduction reads.  Relative bead positions as in
// the integrators (bead 0 the origin, minimum image).
template <int PM, class R>
__global__ void __launch_bounds__(128) k_spring(Dev d)
{
    typedef typename PosT<PM, R>::S PS;
    __shared__ double red[4][kNQ];
    const int cta = blockIdx.x, s = d.icta_sys[cta];
    const DSys S = d.sys[s];
    const int nct = S.icta1 - S.icta0, per = (S.N + nct - 1) / nct;
    const int a0 = (cta - S.icta0) * per, na = max(min(S.N, a0 + per) - a0, 0);
    const size_t G = (size_t)d.G;
    const PS *X = reinterpret_cast<const PS *>(d.x);
    double spring = 0.0;
    // a cell's stored offsets are the physical ones over lam
    const double l2 = (d.npt && d.npt[s].on) ? d.npt[s].lam * d.npt[s].lam : 1.0;
    if (S.P > 1)
        for (int t = threadIdx.x; t < 3 * na; t += blockDim.x) {
            const int c = t / na, i = a0 + (t - c * na);
            const size_t o0 = (size_t)c * G + S.g0 + i;
            const PS x0 = X[o0];
            R prev = 0, sp = 0;
            for (int b = 1; b < S.P; ++b) {
                const R xr = PosT<PM, R>::rel(X[o0 + (size_t)b * S.N], x0, S.box[c], S.fix_scale[c], S.fix_inv[c]);
                const R dd = prev - xr;
                sp = fma(dd, dd, sp);
                prev = xr;
            }
            sp = fma(prev, prev, sp);  // bead P-1 to bead 0 (the origin)
            spring += 0.5 * d.mass_mvv[d.typ[S.g0 + i]] * S.wP * S.wP * (double)sp * l2;
        }
    double acc[kNQ];
    for (int q = 0; q < kNQ; ++q) acc[q] = 0.0;
    acc[Q_SPRING] = warp_sum(spring);
    cta_store_partials(acc, red, d.ipart + (size_t)cta * kNQ);
}

// State upload: positions / velocities of system s from the caller's AoS layout
// [P][N][3] (FP64, copied as is into a staging buffer) to the SoA state, one
// thread per value.  Pair potentials: positions wrapped into the box (mixed
// form: 30-bit fixed point, u = x/L - floor(x/L) rounded half away from zero to
// a multiple of 2^-30); external potentials: as given (FP32 in the mixed form).
template <int PM, class R>
__global__ void k_load_state(Dev d, int s, const double *pos, const double *vel, int near_ref)
{
    const DSys S = d.sys[s];
    const long long n3 = 3LL * S.N * S.P, G = d.G;
    for (long long t = (long long)blockIdx.x * blockDim.x + threadIdx.x; t < n3; t += (long long)gridDim.x * blockDim.x) {
        const long long a = t / 3;
        const int comp = (int)(t - 3 * a);
        const size_t o = (size_t)comp * G + S.g0 + a;
        if (pos) {
            // isothermal-isobaric cell: the state is kept in the reference cell
            const double lam = (d.npt && d.npt[s].on) ? d.npt[s].lam : 1.0;
            const double x = pos[t] / lam, L = S.box[comp];
            // near_ref (the lists exist): between rebuilds a position moves on without
            // wrapping, so that the periodic images of the lists stay valid; the
            // uploaded position is stored as its periodic copy nearest the reference
            // xref, which makes an unchanged state reproduce the stored one and the
            // rebuild test measure the true displacement
            if (PM == PM_FIX) {
                double u = x / L;
                u -= floor(u);
                const long long q = (long long)round(u * (double)(1 << kFixBits));
                int qm = (int)(q & ((1LL << kFixBits) - 1));
                if (near_ref) {
                    const int xr = reinterpret_cast<const int *>(d.xref)[o];
                    qm = (int)((unsigned)xr + (unsigned)fix_minimg((int)((unsigned)qm - (unsigned)xr)));
                }
                reinterpret_cast<int *>(d.x)[o] = qm;
            } else if (PM == PM_BOX64) {
                double w = x - L * floor(x / L);
                if (w >= L || w < 0.0) w = 0.0;
                if (near_ref) {   // w itself unless the reference lies a box length away
                    const double xr = reinterpret_cast<const double *>(d.xref)[o];
                    const double k = rint((xr - w) / L);
                    if (k != 0.0) w += k * L;
                }
                reinterpret_cast<double *>(d.x)[o] = w;
            } else {
                reinterpret_cast<R *>(d.x)[o] = (R)x;
            }
        }
        if (vel) reinterpret_cast<R *>(d.v)[o] = (R)vel[t];
    }
}

void launch_load_state(const Dev &d, const MdLaunch &m, int s, long long n3, const double *pos, const double *vel,
                       int near_ref, cudaStream_t st)
{
    const int grid = (int)std::min<long long>((n3 + 255) / 256, 4096);
    if (!m.pair) {
        if (m.mixed) k_load_state<PM_FREE, float><<<grid, 256, 0, st>>>(d, s, pos, vel, 0);
        else k_load_state<PM_FREE, double><<<grid, 256, 0, st>>>(d, s, pos, vel, 0);
    } else {
        if (m.mixed) k_load_state<PM_FIX, float><<<grid, 256, 0, st>>>(d, s, pos, vel, near_ref);
        else k_load_state<PM_BOX64, double><<<grid, 256, 0, st>>>(d, s, pos, vel, near_ref);
    }
}

// State download: positions (which 0, reported in [0, L) for pair potentials:
// they move unwrapped between list rebuilds), velocities (1) or forces (2) of
// system s into the caller's AoS layout [P][N][3], FP64, one thread per value.
template <int PM, class R>
__global__ void k_store_state(Dev d, int s, int which, double *out)
{
    const DSys S = d.sys[s];
    const long long n3 = 3LL * S.N * S.P, G = d.G;
    for (long long t = (long long)blockIdx.x * blockDim.x + threadIdx.x; t < n3; t += (long long)gridDim.x * blockDim.x) {
        const long long a = t / 3;
        const int comp = (int)(t - 3 * a);
        const size_t o = (size_t)comp * G + S.g0 + a;
        double x;
        if (which == 0 && PM == PM_FIX) {
            const double sc = S.box[comp] / (double)(1 << kFixBits);
            x = (double)(reinterpret_cast<const int *>(d.x)[o] & ((1 << kFixBits) - 1)) * sc;
        } else if (which == 0 && PM == PM_BOX64) {
            const double L = S.box[comp];
            x = reinterpret_cast<const double *>(d.x)[o];
            x = x - L * floor(x / L);
            if (x >= L || x < 0.0) x = 0.0;
        } else {
            const void *src = (which == 0) ? d.x : (which == 1) ? d.v : d.f;
            x = (double)reinterpret_cast<const R *>(src)[o];
        }
        if (which == 0 && PM != PM_FREE && d.npt && d.npt[s].on) x *= d.npt[s].lam;  // physical position
        out[t] = x;
    }
}

void launch_store_state(const Dev &d, const MdLaunch &m, int s, long long n3, int which, double *out, cudaStream_t st)
{
    const int grid = (int)std::min<long long>((n3 + 255) / 256, 4096);
    if (!m.pair) {
        if (m.mixed) k_store_state<PM_FREE, float><<<grid, 256, 0, st>>>(d, s, which, out);
        else k_store_state<PM_FREE, double><<<grid, 256, 0, st>>>(d, s, which, out);
    } else {
        if (m.mixed) k_store_state<PM_FIX, float><<<grid, 256, 0, st>>>(d, s, which, out);
        else k_store_state<PM_BOX64, double><<<grid, 256, 0, st>>>(d, s, which, out);
    }
}

// Before the forces of an uploaded state are computed (pair potentials): the
// packed gather copy pos[cur] of every bead-atom, and a rebuild request for each
// system one of whose bead-atoms lies more than skin/2 from its position at the
// last rebuild -- the test of the integrators; otherwise the lists stay valid.
template <int PM, class R>
__global__ void k_refresh_check(Dev d, int cur)
{
    typedef typename PosT<PM, R>::S PS;
    const size_t G = (size_t)d.G;
    const PS *X = reinterpret_cast<const PS *>(d.x);
    const PS *XR = reinterpret_cast<const PS *>(d.xref);
    const long long tid = (long long)blockIdx.x * blockDim.x + threadIdx.x, nth = (long long)gridDim.x * blockDim.x;
    for (int s = 0; s < d.nsys; ++s) {
        const DSys &S = d.sys[s];
        const long long gn = (long long)S.N * S.P;
        R lim = sizeof(R) == 4 ? (R)S.skin2_f : (R)S.skin2;
        if (d.npt && d.npt[s].on) {  // as the integrator: physical displacement against D^2
            const R l = (R)d.npt[s].lam;
            lim = (sizeof(R) == 4 ? (R)S.npt_d2_f : (R)S.npt_d2) / (l * l);
        }
        bool moved = false;
        for (long long l = ((tid - S.g0) % nth + nth) % nth; l < gn; l += nth) {
            const size_t g = (size_t)(S.g0 + l);
            PS w[3];
            R tot = 0;
            for (int c = 0; c < 3; ++c) {
                w[c] = X[c * G + g];
                const R dc = PosT<PM, R>::diff(w[c], XR[c * G + g], S.fix_scale[c]);
                tot = fma(dc, dc, tot);
            }
            moved |= tot > lim;
            const int t = d.typ[g];
            if (PM == PM_FIX) reinterpret_cast<int4 *>(d.pos[cur])[g] = make_int4((int)w[0], (int)w[1], (int)w[2], t);
            else reinterpret_cast<D4 *>(d.pos[cur])[g] = D4{(double)w[0], (double)w[1], (double)w[2], (double)t};
        }
        if (moved) {
            atomicOr(&d.rflag[cur * d.nsys + s], 1u);
            atomicOr(&d.flag[cur], 1u);
        }
    }
}

void launch_refresh_check(const Dev &d, const MdLaunch &m, int cur, cudaStream_t st)
{
    if (!m.pair) return;
    const int grid = (int)std::min<long long>(((long long)d.G + 255) / 256, 4096);
    if (m.mixed) k_refresh_check<PM_FIX, float><<<grid, 256, 0, st>>>(d, cur);
    else k_refresh_check<PM_BOX64, double><<<grid, 256, 0, st>>>(d, cur);
}

// ---------------------------------------------------------------------------
// Isothermal-isobaric cells: the update of each system's cell at the start of
// step j (cell_update), one thread per system.  Launched before the first step
// of each call; the steps after it get theirs from the step kernel that
// precedes them.
template <bool F32>
__global__ void k_cell(Dev d, int j)
{
    const int s = blockIdx.x * blockDim.x + threadIdx.x;
    if (s >= d.nsys || !d.npt || !d.npt[s].on) return;
    cell_update<F32>(d, s, d.clock[0] * kBlockSteps + j, j & 1);
}

void launch_cell(const Dev &d, int j, bool fp32, cudaStream_t st)
{
    if (fp32)
        k_cell<true><<<(d.nsys + 127) / 128, 128, 0, st>>>(d, j);
    else
        k_cell<false><<<(d.nsys + 127) / 128, 128, 0, st>>>(d, j);
}

// Self-test of the bounded waits: one thread waits on words[0], which nothing
// sets, through the wait of the grid barriers; it gives up after about a second
// and records that in words[1] (not in the context's error word).
__global__ void k_wait_selftest(unsigned *words)
{
    if (blockIdx.x == 0 && threadIdx.x == 0) bounded_wait(words, 0u, words + 1, 1u);
}

__global__ void k_tick(Dev d) { d.clock[0] += 1; }
__global__ void k_setclock(Dev d, long long b) { d.clock[0] = b; }

// ---------------------------------------------------------------------------
// launchers

bool md_supported_P(int P) { return (P >= 1 && P <= 6) || P == 8 || P == 16 || P == 32; }

int integrate_atoms_per_cta(int P, int big) { return P == 1 ? kIntAtomsPerCta : nm_atoms(P, big); }

// integrator launches carry the programmatic-stream-serialisation attribute (the
// kernels wait for the previous launch before reading the state)
template <class K>
static void pdl_launch(K kernel, int grid, int threads, size_t smem, cudaStream_t st, const Dev &d, int j, int cur)
{
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3((unsigned)grid);
    cfg.blockDim = dim3((unsigned)threads);
    cfg.dynamicSmemBytes = smem;
    cfg.stream = st;
    cudaLaunchAttribute at[1];
    at[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
    at[0].val.programmaticStreamSerializationAllowed = 1;
    cfg.attrs = at;
    cfg.numAttrs = 1;
    cudaLaunchKernelEx(&cfg, kernel, d, j, cur);
}

template <int P, int PM, class R>
static void nm_launch(const Dev &d, const MdLaunch &m, int j, int cur, cudaStream_t st)
{
    if (m.nm_big) pdl_launch(k_integrate_nm<P, PM, R, 1>, m.n_icta, nm_threads(P, 1), nm_smem<P, PM, R>(1), st, d, j, cur);
    else pdl_launch(k_integrate_nm<P, PM, R, 0>, m.n_icta, nm_threads(P, 0), nm_smem<P, PM, R>(0), st, d, j, cur);
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
            case 1: pdl_launch(k_integrate<1, PM, R>, m.n_icta, 128, 0, st, d, j, cur); break;
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

void launch_reduce(const Dev &d, const MdLaunch &, int j, int record, cudaStream_t st)
{
    k_reduce<<<d.nsys, 128, 0, st>>>(d, j, record);
}

void launch_centroid(const Dev &d, const MdLaunch &m, int j, int record, int kick, cudaStream_t st)
{
    if (m.n_ccta == 0) return;
    const int g = m.n_ccta, nt = 32 * kCenWarps;
    if (!m.pair) {
        if (m.mixed) k_centroid<PM_FREE, float><<<g, nt, 0, st>>>(d, j, record, kick);
        else k_centroid<PM_FREE, double><<<g, nt, 0, st>>>(d, j, record, kick);
    } else {
        if (m.mixed) k_centroid<PM_FIX, float><<<g, nt, 0, st>>>(d, j, record, kick);
        else k_centroid<PM_BOX64, double><<<g, nt, 0, st>>>(d, j, record, kick);
    }
}

void launch_spring(const Dev &d, const MdLaunch &m, cudaStream_t st)
{
    if (!m.pair) {
        if (m.mixed) k_spring<PM_FREE, float><<<m.n_icta, 128, 0, st>>>(d);
        else k_spring<PM_FREE, double><<<m.n_icta, 128, 0, st>>>(d);
    } else {
        if (m.mixed) k_spring<PM_FIX, float><<<m.n_icta, 128, 0, st>>>(d);
        else k_spring<PM_BOX64, double><<<m.n_icta, 128, 0, st>>>(d);
    }
}

void launch_wait_selftest(unsigned *words, cudaStream_t st) { k_wait_selftest<<<1, 32, 0, st>>>(words); }

void launch_tick(const Dev &d, cudaStream_t st) { k_tick<<<1, 1, 0, st>>>(d); }
void launch_setclock(const Dev &d, long long b, cudaStream_t st) { k_setclock<<<1, 1, 0, st>>>(d, b); }

}  // namespace qtb
