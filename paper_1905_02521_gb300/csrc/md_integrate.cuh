// md_integrate.cuh -- the integrators of the MD hot path (sm_103a), included by
// md.cu: B(dt/2) in bead space, A(dt/2) O(dt) A(dt/2) in normal-mode space (the
// closing B(dt/2) is in the force kernels).
#pragma once
#include "md_kernels.cuh"

namespace qtb {

// ---------------------------------------------------------------------------
// Integrator: B(dt/2) in bead space, then A(dt/2) O A(dt/2) in normal-mode
// space.  Lane 3a + c (a < 10) of a warp takes Cartesian component c of atom
// i with all of its P beads, so that the three components of a bead-atom meet
// in one warp for the neighbour-list displacement test.  Writes the new
// positions to x and (pair potential) to the packed copy pos[cur] that the
// force kernel gathers from, and requests a list rebuild (flag[cur]) when a
// bead-atom has moved more than skin/2 since the last one.

template <int P, int PM, class R>
__global__ void __launch_bounds__(128) k_integrate(Dev d, int j, int cur)
{
    constexpr int UN = (P <= 8) ? P : 1;  // full unroll only for small rings
    typedef typename PosT<PM, R>::S PS;
    __shared__ R Cs[P * P];
    __shared__ double red[4][kNQ];
    const int cta = blockIdx.x;
    const int s = d.icta_sys[cta];
    const DSys S = d.sys[s];
    const bool mine = (S.P == P);  // another instantiation handles the other systems
    if (mine)
        for (int t = threadIdx.x; t < P * P; t += blockDim.x) Cs[t] = reinterpret_cast<const R *>(d.nmC)[S.nm0 + t];
    __syncthreads();
    wait_previous_step();  // as k_integrate_nm
    release_next_step();
    const int N = S.N;
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int aw = lane / 3, c = lane - 3 * aw;
    const int i = (cta - S.icta0) * kIntAtomsPerCta + warp * kIntAtomsPerWarp + aw;
    const bool act = mine && aw < kIntAtomsPerWarp && i < N;
    double acc[kNQ];
    for (int q = 0; q < kNQ; ++q) acc[q] = 0.0;
    double spring = 0.0;
    // the spring energy enters the record of recorded steps only (FP64 is scarce)
    const bool recs = (d.clock[0] * kBlockSteps + j + 1) % d.obs_stride == 0;
    PS *X = reinterpret_cast<PS *>(d.x);
    const size_t G = (size_t)d.G;
    const size_t base = act ? (size_t)c * G + S.g0 + i : 0;
    const float fsc = S.fix_scale[c], finv = S.fix_inv[c];
    // isothermal-isobaric cell (one bead): this step's coefficients from the cell kernel
    const DNpt *NC = (P == 1 && d.npt && d.npt[s].on) ? d.npt + s : nullptr;
    PS x0{};
    R a[P], a0[P];  // bead positions relative to bead 0: new, old
    if (act) {
        R *V = reinterpret_cast<R *>(d.v);
        const R *F = reinterpret_cast<const R *>(d.f);
        const int t = d.typ[S.g0 + i];
        const R hdtm = reinterpret_cast<const R *>(d.hdt_m)[t];
        const R sig = reinterpret_cast<const R *>(d.osig)[s * kMaxTypes + t];
        const double L = S.box[c];
        x0 = X[base];
        R q[P];
        // relative bead positions -> modes
#pragma unroll(UN)
        for (int b = 0; b < P; ++b) {
            a[b] = (b == 0) ? R(0) : PosT<PM, R>::rel(X[base + (size_t)b * N], x0, L, fsc, finv);
            a0[b] = a[b];
        }
#pragma unroll(UN)
        for (int k = 0; k < P; ++k) {
            R u = 0;
#pragma unroll(UN)
            for (int b = 0; b < P; ++b) u = fma(Cs[b * P + k], a[b], u);
            q[k] = u;
        }
        // B: half kick with the current forces, bead velocities -> modes
        if (NC) {  // with the cell's friction: v e1 + (hdt/m) F g1
            const R e1 = sizeof(R) == 4 ? (R)NC->e1f : (R)NC->e1, g1 = sizeof(R) == 4 ? (R)NC->g1f : (R)NC->g1;
            a[0] = fma(V[base], e1, (hdtm * F[base]) * g1);
        } else {
#pragma unroll(UN)
            for (int b = 0; b < P; ++b) a[b] = fma(hdtm, F[base + (size_t)b * N], V[base + (size_t)b * N]);
        }
        R p[P];
#pragma unroll(UN)
        for (int k = 0; k < P; ++k) {
            R u = 0;
#pragma unroll(UN)
            for (int b = 0; b < P; ++b) u = fma(Cs[b * P + k], a[b], u);
            p[k] = u;
        }
        const R *rot = reinterpret_cast<const R *>(d.rot) + 3 * S.rot0;
        const R *eta = reinterpret_cast<const R *>(d.eta) + eta_row(d, j) * d.Dtot + S.dof0;
        const R c1 = sizeof(R) == 4 ? (R)S.c1_f : (R)S.c1;
        if (NC) {
            // one bead in a changing cell: A(dt/2) O(dt) A(dt/2) as displacements in the
            // reference cell (x_ref += v a1, then v' a2: the exact drift of
            // dr/dt = v + v_e r with the cell scaled alike)
            const R a1 = sizeof(R) == 4 ? (R)NC->a1f : (R)NC->a1, a2 = sizeof(R) == 4 ? (R)NC->a2f : (R)NC->a2;
            R pk = p[0];
            R disp = pk * a1;
            pk = fma(c1, pk, sig * eta[(size_t)c * N + i]);
            disp = fma(pk, a2, disp);
            q[0] = q[0] + disp;
            p[0] = pk;
        } else {
#pragma unroll(UN)
            for (int k = 0; k < P; ++k)
                mode_aoa(q[k], p[k], rot[3 * k], rot[3 * k + 1], rot[3 * k + 2], c1, sig * eta[(size_t)(k * 3 + c) * N + i]);
        }
        // modes -> beads
#pragma unroll(UN)
        for (int b = 0; b < P; ++b) {
            R u = 0, w = 0;
#pragma unroll(UN)
            for (int k = 0; k < P; ++k) {
                u = fma(Cs[b * P + k], q[k], u);
                w = fma(Cs[b * P + k], p[k], w);
            }
            a[b] = u;
            V[base + (size_t)b * N] = w;
        }
        if (P > 1 && recs) {
            R sp = 0;
#pragma unroll(UN)
            for (int b = 0; b < P; ++b) {
                R dd = a[b] - a[(b + 1) % P];
                sp = fma(dd, dd, sp);
            }
            spring = 0.5 * d.mass_mvv[t] * S.wP * S.wP * (double)sp;
        }
    }
    // new bead positions: each bead moves by the change of its position relative
    // to bead 0, so that it stays in its own periodic image (after a list rebuild
    // the beads of an atom on the box boundary may be wrapped into different
    // images); with a pair potential also the packed copy and the displacement
    // test (the three components meet through shuffles)
    bool moved = false;
    const int l0 = 3 * aw;
#pragma unroll(UN)
    for (int b = 0; b < P; ++b) {
        R dd = 0;
        if (act) {
            const size_t o = base + (size_t)b * N;
            const PS xn = PosT<PM, R>::add(X[o], a[b] - a0[b], S.box[c], fsc, finv);
            X[o] = xn;
            if (PM != PM_FREE) {
                const size_t g = S.g0 + (size_t)b * N + i;
                reinterpret_cast<PS *>(d.pos[cur])[4 * g + c] = xn;
                const R dc = PosT<PM, R>::diff(xn, reinterpret_cast<const PS *>(d.xref)[o], fsc);
                dd = dc * dc;
            }
        }
        if (PM != PM_FREE) {
            const R tot = __shfl_sync(0xffffffffu, dd, l0 & 31) + __shfl_sync(0xffffffffu, dd, (l0 + 1) & 31) +
                          __shfl_sync(0xffffffffu, dd, (l0 + 2) & 31);
            R lim = sizeof(R) == 4 ? (R)S.skin2_f : (R)S.skin2;
            if (NC) {
                // physical displacement (lam times the reference one) against D^2 (the
                // rest of the skin is the cell kernel's margin for the change of lam
                // since the rebuild; see kNptCellSkin)
                const R l = sizeof(R) == 4 ? (R)NC->lamf : (R)NC->lam;
                lim = (sizeof(R) == 4 ? (R)S.npt_d2_f : (R)S.npt_d2) / (l * l);
            }
            moved |= act && c == 0 && tot > lim;
        }
    }
    if (PM != PM_FREE && __any_sync(0xffffffffu, moved) && lane == 0) {
        atomicOr(&d.rflag[cur * d.nsys + s], 1u);
        atomicOr(&d.flag[cur], 1u);
    }
    if (P > 1 && recs) {
        spring = warp_sum(spring);
        acc[Q_SPRING] = spring;
        if (mine) cta_store_partials(acc, red, d.ipart + (size_t)cta * kNQ);
    }
}

// Ring-polymer integrator for P >= 2 with the normal-mode transforms in shared
// memory.  A CTA takes A atoms of one system, i.e. 3 A columns (component c,
// atom a; col = c A + a) of P beads, V = 3 A P values.  A thread task is MT
// consecutive rows (beads or modes) of one column (register tiling: one shared
// load of a value feeds MT multiply-adds; MT = 1 for P < 8).  Phase 1
// (task = beads): relative bead positions and half-kicked bead velocities
// (B, dt/2) into shared memory.  Phase 2 (task = modes): the forward
// transforms, A(dt/2) O(dt) A(dt/2) of each mode.  Phase 3 (task = beads, the
// mapping of phase 1): back to beads, each bead moved within its own periodic
// image.  Phase 4: spring energy; the tasks of component 0 write the packed
// positions and test each bead-atom's displacement against skin/2.  Every sum
// over beads or modes runs in ascending order, whatever the tiling, so that
// every layout rounds alike.  BIG (large contexts): 32 atoms per CTA, so that
// the 32 threads of a warp read 128 contiguous bytes.
// rows per task (measured on GB300: P = 32 best at 4 rows, 2 or 8 slower; P = 8 at 2)
__host__ __device__ constexpr int nm_rows(int P) { return P >= 16 ? 4 : (P >= 8 ? 2 : 1); }
__host__ __device__ constexpr int nm_atoms(int P, int big) { return big ? 32 : (P >= 16 ? 768 : 192) / (3 * P); }
// compact layout: one thread per task (the transforms are latency-bound chains
// of P multiply-adds; few CTAs per SM at these sizes)
__host__ __device__ constexpr int nm_threads(int P, int big)
{
    return big ? (P >= 8 ? 256 : 128) : (3 * nm_atoms(P, 0) * P / nm_rows(P) + 31) / 32 * 32;
}

template <int P, int PM, class R>
__host__ __device__ constexpr size_t nm_smem(int big)
{
    return (size_t)3 * nm_atoms(P, big) * P * (2 * sizeof(R) + sizeof(typename PosT<PM, R>::S)) +
           (size_t)P * P * sizeof(R) * (nm_rows(P) > 1 ? 2 : 1);
}

// MT consecutive coefficients from shared memory (16-byte aligned when MT = 4)
template <int MT> __device__ __forceinline__ void nm_row(const float *p, float (&c)[MT])
{
    if constexpr (MT == 4) {
        const float4 v = *reinterpret_cast<const float4 *>(p);
        c[0] = v.x; c[1] = v.y; c[2] = v.z; c[3] = v.w;
    } else {
#pragma unroll
        for (int m = 0; m < MT; ++m) c[m] = p[m];
    }
}
template <int MT> __device__ __forceinline__ void nm_row(const double *p, double (&c)[MT])
{
    if constexpr (MT == 4) {
        const double2 a = *reinterpret_cast<const double2 *>(p), b = *reinterpret_cast<const double2 *>(p + 2);
        c[0] = a.x; c[1] = a.y; c[2] = b.x; c[3] = b.y;
    } else {
#pragma unroll
        for (int m = 0; m < MT; ++m) c[m] = p[m];
    }
}

template <int P, int PM, class R, int BIG>
__global__ void __launch_bounds__(nm_threads(P, BIG)) k_integrate_nm(Dev d, int j, int cur)
{
    typedef typename PosT<PM, R>::S PS;
    constexpr int NT = nm_threads(P, BIG), A = nm_atoms(P, BIG), MT = nm_rows(P), NG = P / MT;
    constexpr int COLS = 3 * A, NV = COLS * P, NTASK = NG * COLS, PER = (NTASK + NT - 1) / NT;
    static_assert(P % MT == 0, "rows per task must divide P");
    extern __shared__ __align__(16) unsigned char nsm[];
    R *xs = reinterpret_cast<R *>(nsm);            // [b or k][col]
    R *ps = xs + NV;
    R *Cs = ps + NV;                               // [b][k]
    R *CsT = Cs + P * P;                           // [k][b] (MT > 1)
    PS *xn_s = reinterpret_cast<PS *>(CsT + (MT > 1 ? P * P : 0));  // new positions [b][col]
    __shared__ double red[NT / 32][kNQ];
    const int cta = blockIdx.x;
    const int s = d.icta_sys[cta];
    const DSys S = d.sys[s];
    if (S.P != P) return;  // another instantiation handles this system (uniform over the CTA)
    for (int t = threadIdx.x; t < P * P; t += NT) {
        const R *Cg = reinterpret_cast<const R *>(d.nmC) + S.nm0;
        Cs[t] = Cg[t];
        if (MT > 1) CsT[t] = Cg[(t % P) * P + t / P];  // CsT[k P + b] = C[b][k] (contiguous stores)
    }
    // programmatic dependent launch: the mode matrix above is static; the state is
    // the previous step's (see wait_previous_step)
    wait_previous_step();
    release_next_step();
    const int N = S.N;
    const int i0 = (cta - S.icta0) * A;
    const size_t G = (size_t)d.G;
    PS *X = reinterpret_cast<PS *>(d.x);
    R *V = reinterpret_cast<R *>(d.v);
    const R *F = reinterpret_cast<const R *>(d.f);
    const R *hdt = reinterpret_cast<const R *>(d.hdt_m);
    // isothermal-isobaric cell: it acts on the centroid mode only (the B with its
    // friction needs the velocity and force modes apart: the kicks hdt F / m go to
    // fs, the new-position area, unused until phase 3); stored positions are the
    // physical ones over lam, so the internal modes are taken to physical length
    // with this step's old lam and back with its new one
    const DNpt *NC = (d.npt && d.npt[s].on) ? d.npt + s : nullptr;
    static_assert(sizeof(PS) == sizeof(R), "fs overlays xn_s");
    R *fs = reinterpret_cast<R *>(xn_s);
    // phase 1: loads, then relative positions and B(dt/2) velocities, bead space
    PS xold[PER][MT], x0v[PER];
    R vv[PER][MT], fv[PER][MT], xrel[PER][MT];
    int tt[PER];
#pragma unroll
    for (int u = 0; u < PER; ++u) {
        const int idx = threadIdx.x + u * NT;
        const int g = idx / COLS, col = idx - g * COLS;
        const int c = col / A, i = i0 + (col - c * A);
        x0v[u] = PS(0);
        tt[u] = 0;
#pragma unroll
        for (int m = 0; m < MT; ++m) {
            xold[u][m] = PS(0);
            vv[u][m] = fv[u][m] = R(0);
        }
        if (idx < NTASK && i < N) {
            const size_t o0 = (size_t)c * G + S.g0 + i;
            x0v[u] = X[o0];
            tt[u] = d.typ[S.g0 + i];
#pragma unroll
            for (int m = 0; m < MT; ++m) {
                const size_t o = o0 + (size_t)(g * MT + m) * N;
                xold[u][m] = X[o];
                vv[u][m] = V[o];
                fv[u][m] = F[o];
            }
        }
    }
#pragma unroll
    for (int u = 0; u < PER; ++u) {
        const int idx = threadIdx.x + u * NT;
        if (idx >= NTASK) continue;
        const int g = idx / COLS, col = idx - g * COLS;
        const int c = col / A;
        const R hd = hdt[tt[u]];
#pragma unroll
        for (int m = 0; m < MT; ++m) {
            const int b = g * MT + m;
            const R xr = (b == 0) ? R(0) : PosT<PM, R>::rel(xold[u][m], x0v[u], S.box[c], S.fix_scale[c], S.fix_inv[c]);
            xrel[u][m] = xr;
            xs[b * COLS + col] = xr;
            if (NC) {
                ps[b * COLS + col] = vv[u][m];
                fs[b * COLS + col] = hd * fv[u][m];
            } else {
                ps[b * COLS + col] = fma(hd, fv[u][m], vv[u][m]);
            }
        }
    }
    __syncthreads();
    // phase 2: to modes, A O A per mode
    const R *rot = reinterpret_cast<const R *>(d.rot) + 3 * S.rot0;
    const R *eta = reinterpret_cast<const R *>(d.eta) + eta_row(d, j) * d.Dtot + S.dof0;
    const R c1 = sizeof(R) == 4 ? (R)S.c1_f : (R)S.c1;
    R qv[PER][MT], pm[PER][MT];
#pragma unroll
    for (int u = 0; u < PER; ++u) {
        const int idx = threadIdx.x + u * NT;
        const int g = idx / COLS, col = idx - g * COLS;
        const int c = col / A, i = i0 + (col - c * A);
        R noise[MT];
#pragma unroll
        for (int m = 0; m < MT; ++m) noise[m] = R(0);
        if (idx < NTASK && i < N) {
            const R sig = reinterpret_cast<const R *>(d.osig)[s * kMaxTypes + tt[u]];
#pragma unroll
            for (int m = 0; m < MT; ++m) noise[m] = sig * eta[(size_t)((g * MT + m) * 3 + c) * N + i];
        }
        R q[MT], p[MT];
#pragma unroll
        for (int m = 0; m < MT; ++m) q[m] = p[m] = R(0);
        if (idx < NTASK && !NC) {
#pragma unroll 8
            for (int b = 0; b < P; ++b) {
                const R xv = xs[b * COLS + col], pv = ps[b * COLS + col];
                R cf[MT];
                nm_row<MT>(Cs + b * P + g * MT, cf);
#pragma unroll
                for (int m = 0; m < MT; ++m) {
                    q[m] = fma(cf[m], xv, q[m]);
                    p[m] = fma(cf[m], pv, p[m]);
                }
            }
#pragma unroll
            for (int m = 0; m < MT; ++m) {
                const int k = g * MT + m;
                mode_aoa(q[m], p[m], rot[3 * k], rot[3 * k + 1], rot[3 * k + 2], c1, noise[m]);
            }
        } else if (idx < NTASK) {
            R pf[MT];
#pragma unroll
            for (int m = 0; m < MT; ++m) pf[m] = R(0);
#pragma unroll 8
            for (int b = 0; b < P; ++b) {
                const R xv = xs[b * COLS + col], pv = ps[b * COLS + col], fb = fs[b * COLS + col];
                R cf[MT];
                nm_row<MT>(Cs + b * P + g * MT, cf);
#pragma unroll
                for (int m = 0; m < MT; ++m) {
                    q[m] = fma(cf[m], xv, q[m]);
                    p[m] = fma(cf[m], pv, p[m]);
                    pf[m] = fma(cf[m], fb, pf[m]);
                }
            }
            const bool f32 = sizeof(R) == 4;
            const R e1 = f32 ? (R)NC->e1f : (R)NC->e1, g1 = f32 ? (R)NC->g1f : (R)NC->g1;
            const R a1 = f32 ? (R)NC->a1f : (R)NC->a1, a2 = f32 ? (R)NC->a2f : (R)NC->a2;
            const R lo = f32 ? (R)NC->lam_oldf : (R)NC->lam_old, il = f32 ? (R)NC->inv_lamf : (R)NC->inv_lam;
#pragma unroll
            for (int m = 0; m < MT; ++m) {
                const int k = g * MT + m;
                if (k == 0) {
                    // centroid: B with the cell's friction, then A O A as a drift in the
                    // reference cell (the one-bead integrator's factors)
                    R pk = fma(p[m], e1, pf[m] * g1);
                    R disp = pk * a1;
                    pk = fma(c1, pk, noise[m]);
                    disp = fma(pk, a2, disp);
                    q[m] = q[m] + disp;
                    p[m] = pk;
                } else {
                    R qk = q[m] * lo;
                    p[m] = p[m] + pf[m];
                    mode_aoa(qk, p[m], rot[3 * k], rot[3 * k + 1], rot[3 * k + 2], c1, noise[m]);
                    q[m] = qk * il;
                }
            }
        }
#pragma unroll
        for (int m = 0; m < MT; ++m) {
            qv[u][m] = q[m];
            pm[u][m] = p[m];
        }
    }
    __syncthreads();
#pragma unroll
    for (int u = 0; u < PER; ++u) {
        const int idx = threadIdx.x + u * NT;
        if (idx >= NTASK) continue;
        const int g = idx / COLS, col = idx - g * COLS;
#pragma unroll
        for (int m = 0; m < MT; ++m) {
            xs[(g * MT + m) * COLS + col] = qv[u][m];
            ps[(g * MT + m) * COLS + col] = pm[u][m];
        }
    }
    __syncthreads();
    // phase 3: back to beads (positions stay in each bead's own image)
    const R *Cb = (MT > 1) ? CsT : Cs;  // C[b][k] at CsT[k P + b] (tiled) or Cs[b P + k]
#pragma unroll
    for (int u = 0; u < PER; ++u) {
        const int idx = threadIdx.x + u * NT;
        if (idx >= NTASK) continue;
        const int g = idx / COLS, col = idx - g * COLS;
        R x[MT], w[MT];
#pragma unroll
        for (int m = 0; m < MT; ++m) x[m] = w[m] = R(0);
#pragma unroll 8
        for (int k = 0; k < P; ++k) {
            const R qk = xs[k * COLS + col], pk = ps[k * COLS + col];
            R cf[MT];
            if (MT > 1) {
                nm_row<MT>(Cb + k * P + g * MT, cf);
            } else {
#pragma unroll
                for (int m = 0; m < MT; ++m) cf[m] = Cb[(g * MT + m) * P + k];
            }
#pragma unroll
            for (int m = 0; m < MT; ++m) {
                x[m] = fma(cf[m], qk, x[m]);
                w[m] = fma(cf[m], pk, w[m]);
            }
        }
#pragma unroll
        for (int m = 0; m < MT; ++m) {
            qv[u][m] = x[m];  // new relative position
            pm[u][m] = w[m];  // new velocity
        }
    }
    __syncthreads();
#pragma unroll
    for (int u = 0; u < PER; ++u) {
        const int idx = threadIdx.x + u * NT;
        if (idx >= NTASK) continue;
        const int g = idx / COLS, col = idx - g * COLS;
        const int c = col / A, i = i0 + (col - c * A);
#pragma unroll
        for (int m = 0; m < MT; ++m) {
            const int b = g * MT + m;
            xs[b * COLS + col] = qv[u][m];
            if (i < N) {
                const size_t o = (size_t)c * G + S.g0 + (size_t)b * N + i;
                V[o] = pm[u][m];
                const PS xn = PosT<PM, R>::add(xold[u][m], qv[u][m] - xrel[u][m], S.box[c], S.fix_scale[c], S.fix_inv[c]);
                X[o] = xn;
                xn_s[b * COLS + col] = xn;
            }
        }
    }
    __syncthreads();
    // phase 4: spring energy; packed positions and displacement test per bead-atom
    double spring = 0.0;
    const bool recs = (d.clock[0] * kBlockSteps + j + 1) % d.obs_stride == 0;  // spring only where recorded
    bool moved = false;
    R lim = sizeof(R) == 4 ? (R)S.skin2_f : (R)S.skin2;
    double l2 = 1.0;  // physical length squared over stored (cell)
    if (NC) {
        // physical displacement against D^2 (see k_integrate)
        const R l = sizeof(R) == 4 ? (R)NC->lamf : (R)NC->lam;
        lim = (sizeof(R) == 4 ? (R)S.npt_d2_f : (R)S.npt_d2) / (l * l);
        l2 = NC->lam * NC->lam;
    }
#pragma unroll
    for (int u = 0; u < PER; ++u) {
        const int idx = threadIdx.x + u * NT;
        if (idx >= NTASK) continue;
        const int g = idx / COLS, col = idx - g * COLS;
        const int c = col / A, a = col - c * A, i = i0 + a;
        if (i >= N) continue;
#pragma unroll
        for (int m = 0; m < MT; ++m) {
            const int b = g * MT + m;
            const R dx = xs[b * COLS + col] - xs[((b + 1) % P) * COLS + col];
            if (recs) spring += 0.5 * d.mass_mvv[tt[u]] * S.wP * S.wP * (double)(dx * dx) * l2;
            if (PM != PM_FREE && c == 0) {
                const size_t gg = S.g0 + (size_t)b * N + i;
                const PS *XR = reinterpret_cast<const PS *>(d.xref);
                R tot = 0;
                PS w3[3];
#pragma unroll
                for (int cc = 0; cc < 3; ++cc) {
                    w3[cc] = xn_s[b * COLS + cc * A + a];
                    const R dc = PosT<PM, R>::diff(w3[cc], XR[(size_t)cc * G + gg], S.fix_scale[cc]);
                    tot = fma(dc, dc, tot);
                }
                moved |= tot > lim;
                if (PM == PM_FIX) {
                    int4 *pk = reinterpret_cast<int4 *>(d.pos[cur]);
                    pk[gg] = make_int4((int)w3[0], (int)w3[1], (int)w3[2], tt[u]);
                } else {
                    D4 *pk = reinterpret_cast<D4 *>(d.pos[cur]);
                    pk[gg] = D4{(double)w3[0], (double)w3[1], (double)w3[2], (double)tt[u]};
                }
            }
        }
    }
    if (PM != PM_FREE && __syncthreads_or(moved) && threadIdx.x == 0) {
        atomicOr(&d.rflag[cur * d.nsys + s], 1u);
        atomicOr(&d.flag[cur], 1u);
    }
    if (recs) {
        double acc[kNQ];
        for (int q = 0; q < kNQ; ++q) acc[q] = 0.0;
        acc[Q_SPRING] = warp_sum(spring);
        cta_store_partials(acc, red, d.ipart + (size_t)cta * kNQ);
    }
}

}  // namespace qtb
