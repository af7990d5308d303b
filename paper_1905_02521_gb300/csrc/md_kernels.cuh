// md_kernels.cuh -- device code of the MD hot path (sm_103a) shared by the
// integrators (md_integrate.cuh, md.cu) and the step kernel (md_step8.cu,
// md_step16.cu and md_step32.cu: 8, 16 and 32 lanes per bead-atom, compiled in
// parallel): position representations, reductions, the grid barrier, the mode
// propagator, the list rebuild, the pair force and the step kernel itself.
//
// Eq. 4: every bead feels -(1/P) grad V of its own replica plus the ring
// springs; the springs are integrated exactly in normal-mode space (Sec. 2.3,
// Eq. 11 with the physical force entering through the B kicks).  Eq. 8: the
// Langevin O step carries the coloured random force.  Eq. 5: primitive energy
// estimator, accumulated in FP64.
//
// Mixed form: positions in 30-bit fixed point per box edge (exact integer
// displacements, periodic wrap by masking), FP32 arithmetic, per-atom forces
// summed in float-float (error-free TwoSum per lane and across the warp), so
// that the only FP32 errors left are those of the individual pair terms.
//
// Pair forces come from Verlet neighbour lists (every pair within r_cut +
// skin at the last rebuild, with its periodic image).  Positions move
// continuously between rebuilds and are wrapped into the box only when the
// lists are rebuilt, which happens when some bead-atom has moved more than
// skin/2 since the last one: then no pair outside a list can have come within
// r_cut.  For one-bead systems the force kernel also carries out the first
// half of the next step (B, A, O, A), so that a step is one launch.
#pragma once
#include <algorithm>
#include <climits>
#include <type_traits>

#include "qtb_dev.cuh"
#include "qtb_kernels.cuh"

namespace qtb {

struct alignas(32) D4 {  // packed FP64 position + type of one cell slot
    double x, y, z, w;
};

// ---------------------------------------------------------------------------
// position storage

template <int PM, class R> struct PosT;

// rel: minimum-image difference; add: move (no wrap, see above); diff: plain
// difference in A (displacement since the last rebuild)
template <class R> struct PosT<PM_BOX64, R> {  // FP64 A, in [0, L) at each rebuild
    typedef double S;
    __device__ static R rel(S a, S b, double L, float, float)
    {
        double d = a - b;
        return (R)(d - L * rint(d / L));
    }
    __device__ static S add(S a, R delta, double, float, float) { return a + (double)delta; }
    __device__ static R diff(S a, S b, float) { return (R)(a - b); }
    __device__ static S wrap(S x, double L)
    {
        x -= L * floor(x / L);
        return (x >= L || x < 0.0) ? 0.0 : x;
    }
};

template <class R> struct PosT<PM_FIX, R> {  // 30-bit fixed point per box edge, in [0, 2^30) at each rebuild
    typedef int S;
    __device__ static R rel(S a, S b, double, float scale, float) { return (R)fix_minimg(a - b) * (R)scale; }
    __device__ static S add(S a, R delta, double, float, float inv)
    {
        const int dq = __float2int_rn((float)delta * inv);
        return (int)((unsigned)a + (unsigned)dq);
    }
    __device__ static R diff(S a, S b, float scale) { return (R)(int)((unsigned)a - (unsigned)b) * (R)scale; }
    __device__ static S wrap(S x, double) { return x & (int)((1u << kFixBits) - 1u); }
};

template <class R> struct PosT<PM_FREE, R> {  // unbounded (external potentials)
    typedef R S;
    __device__ static R rel(S a, S b, double, float, float) { return a - b; }
    __device__ static S add(S a, R delta, double, float, float) { return a + delta; }
    __device__ static R diff(S a, S b, float) { return a - b; }
    __device__ static S wrap(S x, double) { return x; }
};

__device__ __forceinline__ double warp_sum(double v)
{
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    return v;
}
__device__ __forceinline__ float warp_sum(float v)
{
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    return v;
}

// error-free sum: s + e = a + b exactly (Knuth's TwoSum)
__device__ __forceinline__ void two_sum(float a, float b, float &s, float &e)
{
    s = __fadd_rn(a, b);
    const float z = __fsub_rn(s, a);
    e = __fadd_rn(__fsub_rn(a, __fsub_rn(s, z)), __fsub_rn(b, z));
}

// float-float accumulator
struct FF {
    float hi, lo;
    __device__ void add(float x)
    {
        float s, e;
        two_sum(hi, x, s, e);
        hi = s;
        lo = __fadd_rn(lo, e);
    }
    __device__ void warp_reduce()
    {
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) {
            const float oh = __shfl_xor_sync(0xffffffffu, hi, o), ol = __shfl_xor_sync(0xffffffffu, lo, o);
            float s, e;
            two_sum(hi, oh, s, e);
            hi = s;
            lo = __fadd_rn(__fadd_rn(lo, ol), e);
        }
    }
    // sum over aligned groups of W lanes (W a power of two <= 32)
    template <int W> __device__ void group_reduce()
    {
#pragma unroll
        for (int o = W / 2; o > 0; o >>= 1) {
            const float oh = __shfl_xor_sync(0xffffffffu, hi, o), ol = __shfl_xor_sync(0xffffffffu, lo, o);
            float s, e;
            two_sum(hi, oh, s, e);
            hi = s;
            lo = __fadd_rn(__fadd_rn(lo, ol), e);
        }
    }
    __device__ float value() const { return __fadd_rn(hi, lo); }
    // add another float-float value (bh + bl)
    __device__ void add_ff(float bh, float bl)
    {
        float s, e;
        two_sum(hi, bh, s, e);
        hi = s;
        lo = __fadd_rn(__fadd_rn(lo, bl), e);
    }
    // sum over the lanes l, l ^ W, l ^ 2W, ... (W a power of two <= 16): lane l < W
    // ends with the sum over its residue class mod W
    template <int W> __device__ void across_groups()
    {
#pragma unroll
        for (int o = 16; o >= W; o >>= 1)
            add_ff(__shfl_xor_sync(0xffffffffu, hi, o), __shfl_xor_sync(0xffffffffu, lo, o));
    }
};

// plain accumulator with the same interface (FP64 form)
struct DD {
    double hi;
    __device__ void add(double x) { hi += x; }
    __device__ void warp_reduce() { hi = warp_sum(hi); }
    template <int W> __device__ void group_reduce()
    {
#pragma unroll
        for (int o = W / 2; o > 0; o >>= 1) hi += __shfl_xor_sync(0xffffffffu, hi, o);
    }
    __device__ double value() const { return hi; }
};

template <int W, class T> __device__ __forceinline__ T group_sum(T v)
{
#pragma unroll
    for (int o = W / 2; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    return v;
}

// CTA-wide sum of kNQ doubles held by lane 0 of each warp into out[0..kNQ)
static __device__ void cta_store_partials(const double *acc, double (*red)[kNQ], double *out)
{
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31, nw = blockDim.x >> 5;
    if (lane == 0)
        for (int q = 0; q < kNQ; ++q) red[warp][q] = acc[q];
    __syncthreads();
    if (threadIdx.x < kNQ) {
        double s = 0.0;
        for (int w = 0; w < nw; ++w) s += red[w][threadIdx.x];
        out[threadIdx.x] = s;
    }
}

// FP32 form of the above for the list force kernel: the float-float sums of a
// CTA's bead-atoms, stored as (hi, lo) pairs in out[0..kNQ).  The potential
// energy and virial halves (en, w*) count on the lanes `lead` (one per
// bead-atom), the kinetic energy kc + kl and momentum mc + ml of component c on
// lane c of each LPA-lane group.  red is the CTA's [warps][kNQ] scratch (8 bytes
// an entry).
template <int LPA>
static __device__ void cta_store_partials_ff(bool lead, float en, float w0, float w1, float w2, float w3, float w4,
                                             float w5, float kc, float kl, float mc, float ml, double (*red)[kNQ],
                                             float2 *out)
{
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31, nw = blockDim.x >> 5;
    static_assert(kNQ == 16 && Q_X2 == 12 && Q_MOM + 2 < 13, "slots 13 and 14 must be free");
    float2 (*rf)[kNQ] = reinterpret_cast<float2 (*)[kNQ]>(red);
    const float h[7] = {en, w0, w1, w2, w3, w4, w5};
    constexpr int slot[7] = {Q_V, Q_VIR + 0, Q_VIR + 1, Q_VIR + 2, Q_VIR + 3, Q_VIR + 4, Q_VIR + 5};
#pragma unroll
    for (int k = 0; k < 7; ++k) {
        FF a{lead ? 0.5f * h[k] : 0.f, 0.f};  // pairs are counted from both ends
        a.template across_groups<LPA>();
        if (lane == 0) rf[warp][slot[k]] = make_float2(a.hi, a.lo);
    }
    FF K{kc, kl}, M{mc, ml};
    K.template across_groups<LPA>();
    M.template across_groups<LPA>();
    // component c of the warp's kinetic energy goes to slot Q_K (c = 0) or to the
    // free slots 13 and 14, joined below
    if (lane < 3) {
        rf[warp][lane == 0 ? Q_K : 12 + lane] = make_float2(K.hi, K.lo);
        rf[warp][Q_MOM + lane] = make_float2(M.hi, M.lo);
    }
    if (lane == 0) rf[warp][Q_SPRING] = rf[warp][Q_X2] = rf[warp][15] = make_float2(0.f, 0.f);
    __syncthreads();
    if (threadIdx.x < kNQ) {
        const int q = threadIdx.x;
        FF t{0.f, 0.f};
        if (q != 13 && q != 14)
            for (int w = 0; w < nw; ++w) t.add_ff(rf[w][q].x, rf[w][q].y);
        if (q == Q_K)
            for (int w = 0; w < nw; ++w) {
                t.add_ff(rf[w][13].x, rf[w][13].y);
                t.add_ff(rf[w][14].x, rf[w][14].y);
            }
        out[q] = make_float2(t.hi, t.lo);
    }
}

// Grid-wide barrier of a cooperative launch (all CTAs co-resident): arrival
// counter bar[0] and generation bar[1].  The wait is bounded: after about a
// second it records ERR_TIMEOUT_BAR and lets the CTA go on (the results of
// that launch are then void, the host reports QTB_ERR_TIMEOUT).  Called by
// all threads of every CTA.
// Bounded wait: spin while *word == value, for at most about a second of
// device time (%globaltimer, ns; a spin count as a second bound).  Gives up at
// once when another wait of the launch already gave up (timeout bit `bit` set in
// *err).  Returns false when it gave up, after setting that bit.
__device__ __forceinline__ unsigned long long device_ns()
{
    unsigned long long t;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
    return t;
}
static __device__ bool bounded_wait(volatile const unsigned *word, unsigned value, unsigned *err, unsigned bit)
{
    const unsigned long long t0 = device_ns();
    long long spins = 0;
    while (*word == value) {
        ++spins;
        if ((spins & 255) == 0 &&
            (device_ns() - t0 > 1000000000ull || spins > (1LL << 26) || (*(volatile const unsigned *)err & bit))) {
            atomicOr(err, bit);
            return false;
        }
        __nanosleep(32);
    }
    return true;
}

static __device__ void grid_barrier(const Dev &d)
{
    __syncthreads();
    if (threadIdx.x == 0) {
        volatile unsigned *gen = d.gbar + 1;
        const unsigned g0 = *gen;
        __threadfence();
        const unsigned arrived = atomicAdd(d.gbar, 1u);
        if (arrived == gridDim.x * gridDim.y - 1u) {
            d.gbar[0] = 0u;
            __threadfence();
            atomicAdd(d.gbar + 1, 1u);
        } else {
            // bounded; after one timeout every later barrier of the launch gives up at once
            bounded_wait(gen, g0, d.err, (unsigned)ERR_TIMEOUT_BAR);
        }
        __threadfence();
    }
    __syncthreads();
}

// One normal mode: A(dt/2) (exact free ring-polymer rotation, (cos, sin/w,
// -w sin) = (cs, sw, ws); for the centroid (1, dt/2, 0) a drift), O(dt) with
// the random kick `noise` = sqrt((1 - c1^2)/m) eta, A(dt/2).  (q, p) in place.
// Shared by the integrator and the fused force epilogue, with every
// multiply-add written out (this file is compiled without contraction), so
// that both round alike.
template <class R>
__device__ __forceinline__ void mode_aoa(R &q, R &p, R cs, R sw, R ws, R c1, R noise)
{
    const R qn = fma(p, sw, q * cs);
    R pn = fma(p, cs, q * ws);
    pn = fma(c1, pn, noise);
    q = fma(pn, sw, qn * cs);
    p = fma(pn, cs, qn * ws);
}

// Programmatic dependent launch of consecutive step launches: a launch may
// begin (its CTAs become resident and stage the pair table) while the previous
// one drains; before reading anything a step writes it waits here for the
// previous launch to complete, and it lets the next launch begin once its own
// list rebuild is over.  Measured on the 8000-ion crystal: 14.0 us per step
// instead of 14.8.
__device__ __forceinline__ void wait_previous_step() { asm volatile("griddepcontrol.wait;" ::: "memory"); }
__device__ __forceinline__ void release_next_step() { asm volatile("griddepcontrol.launch_dependents;" ::: "memory"); }

// ---------------------------------------------------------------------------
// List rebuild: three phases of the cooperative step kernel, separated by grid
// barriers, run only when flag[cur] is set, and then only for the systems
// whose own request is set (rflag[cur]; every system with rebuild scope 1):
// each system rebuilds on its own schedule, so that a system of a batch runs
// exactly as it would alone.
// bin_phase wraps the positions into the box (x, its packed copy pos[cur] and
// the reference xref) and bins them into cells >= (r_cut + skin)/2 with atomic
// slots; sort_phase puts each cell's slots in bead-atom order (so that every
// list, and every later sum, has a fixed order); build_cell scans the 5^3
// stencil of one cell.

// one bead-atom g of replica R: wrap, pack, bin
template <int PM>
__device__ __forceinline__ void bin_one(const Dev &d, int cur, long long g, const DRep &R)
{
    typedef typename PosT<PM, double>::S PS;
    typedef typename std::conditional<PM == PM_FIX, int4, D4>::type E4;
    const size_t G = (size_t)d.G;
    PS *X = reinterpret_cast<PS *>(d.x);
    PS *XR = reinterpret_cast<PS *>(d.xref);
    PS w[3];
    int cc[3];
    for (int c = 0; c < 3; ++c) {
        const double L = R.box[c];
        const int ncc = R.nc[c];
        const PS xw = PosT<PM, double>::wrap(X[c * G + g], L);
        X[c * G + g] = xw;
        XR[c * G + g] = xw;
        w[c] = xw;
        int v;
        if (PM == PM_FIX) v = (int)(((unsigned long long)(unsigned)xw * (unsigned)ncc) >> kFixBits);
        else v = (int)floor((double)xw / L * ncc);
        cc[c] = min(max(v, 0), ncc - 1);
    }
    E4 p;
    p.x = w[0]; p.y = w[1]; p.z = w[2];
    if (PM == PM_FIX) p.w = d.typ[g]; else p.w = (double)d.typ[g];
    reinterpret_cast<E4 *>(d.pos[cur])[g] = p;
    const int cell = R.cell0 + cc[0] + R.nc[0] * (cc[1] + R.nc[1] * cc[2]);
    const int slot = atomicAdd(&d.cnt[cell], 1);
    if (slot < d.cap)
        d.cidx[(size_t)cell * d.cap + slot] = (int)g;
    else
        atomicOr(d.err, (unsigned)ERR_OVERFLOW);
}

// the bead-atoms of the systems that requested a rebuild (rflag[cur]); the
// others keep their lists, positions and reference positions
template <int PM>
__device__ void bin_phase(const Dev &d, int cur)
{
    const unsigned *rf = d.rflag + cur * d.nsys;
    const long long tid = (long long)blockIdx.x * blockDim.x + threadIdx.x, nth = (long long)gridDim.x * blockDim.x;
    for (int s = 0; s < d.nsys; ++s) {
        if (!d.rebuild_all && rf[s] == 0u) continue;
        const DSys &S = d.sys[s];
        const long long gn = (long long)S.N * S.P;
        // the grid-stride mapping of all bead-atoms, restricted to this system's range
        // (consecutive systems land on different threads)
        for (long long l = ((tid - S.g0) % nth + nth) % nth; l < gn; l += nth)
            bin_one<PM>(d, cur, S.g0 + l, d.rep[S.rep0 + (int)(l / S.N)]);
    }
}

// one cell by one warp: slots in bead-atom order, packed positions
template <int PM>
__device__ __forceinline__ void sort_cell(const Dev &d, int cell, int *kw, int lane)
{
    const size_t G = (size_t)d.G;
    const int n = min(d.cnt[cell], d.cap);
    for (int e = lane; e < n; e += 32) kw[e] = d.cidx[(size_t)cell * d.cap + e];
    __syncwarp();
    const int g0 = d.rep[d.cell_rep[cell]].g0;
    for (int e = lane; e < n; e += 32) {
        const int g = kw[e];
        int rank = 0;
        for (int t = 0; t < n; ++t) rank += (kw[t] < g) ? 1 : 0;
        const size_t o = (size_t)cell * d.cap + rank;
        d.cidx[o] = g;
        if (PM == PM_FIX) {
            const int *X = reinterpret_cast<const int *>(d.x);
            reinterpret_cast<int4 *>(d.cpos)[o] = make_int4(X[g], X[G + g], X[2 * G + g], g - g0);
        } else {
            const double *X = reinterpret_cast<const double *>(d.x);
            reinterpret_cast<D4 *>(d.cpos)[o] = D4{X[g], X[G + g], X[2 * G + g], (double)(g - g0)};
        }
    }
    __syncwarp();
    if (lane == 0) {
        d.ccount[cell] = n;
        d.cnt[cell] = 0;
    }
}

// one warp per cell of the requesting systems; keys: kMaxCellCap ints of shared
// memory per warp
template <int PM>
__device__ void sort_phase(const Dev &d, int cur, int *keys)
{
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31, nw = blockDim.x >> 5;
    int *kw = keys + warp * kMaxCellCap;
    const unsigned *rf = d.rflag + cur * d.nsys;
    const int wg = blockIdx.x * nw + warp, W = gridDim.x * nw;
    for (int s = 0; s < d.nsys; ++s) {
        if (!d.rebuild_all && rf[s] == 0u) continue;  // uniform over the grid
        const int c0 = d.sys[s].cell0;
        for (int cell = c0 + ((wg - c0) % W + W) % W; cell < d.sys[s].cell1; cell += W) sort_cell<PM>(d, cell, kw, lane);
    }
}

// List build.  One CTA per home cell: its warps stage the stencil cells
// (sorted slots; image shift added, fixed point + m 2^30 in wrapping int32
// arithmetic; entry word = local index | image bits) chunk by chunk, and for
// each chunk every warp takes one home bead-atom at a time, scans the flat
// staged array and appends the entries within r_cut + skin to the bead-atom's
// list, so that a list is in stencil scan order.
constexpr int kStencilHalf = 2;
constexpr int kStencil = (2 * kStencilHalf + 1) * (2 * kStencilHalf + 1) * (2 * kStencilHalf + 1);

// shared memory of build_cell (besides the staging chunk)
struct BuildSmem {
    int soff[kStencil + 1], scell[kStencil], simg[kStencil][3];
    int scount[kMaxCellCap];
};

template <int PM, class R>
__device__ void build_cell(const Dev &d, R rc2, R rl2, int cell, void *stage_mem, BuildSmem &B)
{
    typedef typename std::conditional<PM == PM_FIX, int4, D4>::type E4;
    constexpr int SH = kStencilHalf, SW = 2 * kStencilHalf + 1;
    int *soff = B.soff, *scell = B.scell, *scount = B.scount;
    int (*simg)[3] = B.simg;
    E4 *stage = reinterpret_cast<E4 *>(stage_mem);
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31, nwarp = blockDim.x >> 5;
    __syncthreads();  // the previous cell of this CTA is done with the shared memory
    const int cnt = d.ccount[cell];
    if (cnt == 0) return;  // uniform over the CTA
    const DRep RP = d.rep[d.cell_rep[cell]];
    const int lc = cell - RP.cell0;
    const int cx = lc % RP.nc[0], cy = (lc / RP.nc[0]) % RP.nc[1], cz = lc / (RP.nc[0] * RP.nc[1]);
    for (int t = threadIdx.x; t < kStencil; t += blockDim.x) {
        const int ox = t % SW - SH, oy = (t / SW) % SW - SH, oz = t / (SW * SW) - SH;
        int ux = cx + ox, uy = cy + oy, uz = cz + oz;
        const int mx = (int)floor_div(ux, RP.nc[0]), my = (int)floor_div(uy, RP.nc[1]), mz = (int)floor_div(uz, RP.nc[2]);
        ux -= mx * RP.nc[0]; uy -= my * RP.nc[1]; uz -= mz * RP.nc[2];
        const int nc = RP.cell0 + ux + RP.nc[0] * (uy + RP.nc[1] * uz);
        scell[t] = nc;
        simg[t][0] = mx; simg[t][1] = my; simg[t][2] = mz;
        soff[t + 1] = d.ccount[nc];
    }
    __syncthreads();
    if (warp == 0) {  // exclusive scan of the stencil counts (<= 128 entries)
        int v[4], run = 0;
#pragma unroll
        for (int k = 0; k < 4; ++k) {
            const int t = lane * 4 + k;
            v[k] = (t < kStencil) ? soff[t + 1] : 0;
            run += v[k];
        }
        int incl = run;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const int y = __shfl_up_sync(0xffffffffu, incl, o);
            if (lane >= o) incl += y;
        }
        int base = incl - run;
#pragma unroll
        for (int k = 0; k < 4; ++k) {
            const int t = lane * 4 + k;
            if (t < kStencil) soff[t] = base;
            base += v[k];
            if (t == kStencil - 1) soff[kStencil] = base;
        }
    }
    __syncthreads();
    // the neighbourhood streams through shared memory in chunks of stage_cap
    // entries (a multiple of 64); each home slot's list grows chunk by chunk
    const int total = soff[kStencil];
    const int CH = d.stage_cap;
    for (int t = threadIdx.x; t < cnt; t += blockDim.x) scount[t] = 0;
    // physical distances (isothermal-isobaric: the reference cell scaled by lam)
    const R lam = (d.npt && d.npt[RP.sys].on) ? (R)d.npt[RP.sys].lam : R(1);
    const R sx = (R)RP.fix_scale[0] * lam, sy = (R)RP.fix_scale[1] * lam, sz = (R)RP.fix_scale[2] * lam;
    const unsigned lt = (1u << lane) - 1u;
    const int maxnb = d.maxnb;
    // pass 0 lists the entries within r_cut, pass 1 those of the skin shell, so
    // that the shell entries close every list (the force loop can skip them)
    for (int pass = 0; pass < 2; ++pass)
    for (int c0 = 0; c0 < total; c0 += CH) {
        const int cn = min(CH, total - c0);
        const int padded = (cn + 63) & ~63;
        __syncthreads();  // the previous chunk is scanned
        // flat staging: every thread first issues all of its (independent) loads,
        // then shifts by the image and stores
        constexpr int U = 4;
        for (int base = 0; base < cn; base += U * (int)blockDim.x) {
            E4 buf[U];
            int tcell[U], dst[U];
#pragma unroll
            for (int u = 0; u < U; ++u) {
                const int el = base + u * (int)blockDim.x + (int)threadIdx.x;
                dst[u] = -1;
                tcell[u] = 0;
                if (el < cn) {
                    const int e = c0 + el;
                    int lo = 0, hi = kStencil - 1;  // stencil cell t with soff[t] <= e < soff[t+1]
                    while (lo < hi) {
                        const int mid = (lo + hi + 1) >> 1;
                        if (soff[mid] <= e) lo = mid; else hi = mid - 1;
                    }
                    tcell[u] = lo;
                    dst[u] = el;
                    buf[u] = reinterpret_cast<const E4 *>(d.cpos)[(size_t)scell[lo] * d.cap + (e - soff[lo])];
                }
            }
#pragma unroll
            for (int u = 0; u < U; ++u) {
                if (dst[u] < 0) continue;
                E4 p = buf[u];
                const int t = tcell[u];
                const int mx = simg[t][0], my = simg[t][1], mz = simg[t][2];
                const unsigned ib = ((unsigned)(mx & 3) << 26) | ((unsigned)(my & 3) << 28) | ((unsigned)(mz & 3) << 30);
                if (PM == PM_FIX) {
                    p.x = (int)((unsigned)p.x + (unsigned)mx * (1u << kFixBits));
                    p.y = (int)((unsigned)p.y + (unsigned)my * (1u << kFixBits));
                    p.z = (int)((unsigned)p.z + (unsigned)mz * (1u << kFixBits));
                    p.w = (int)((unsigned)p.w | ib);
                } else {
                    p.x += mx * RP.box[0];
                    p.y += my * RP.box[1];
                    p.z += mz * RP.box[2];
                    p.w = (double)((unsigned)p.w | ib);
                }
                stage[dst[u]] = p;
            }
        }
        // sentinel entries far outside the list radius pad the scan to a multiple of 64
        for (int e = cn + threadIdx.x; e < padded; e += blockDim.x) {
            if (PM == PM_FIX) reinterpret_cast<int4 *>(stage)[e] = make_int4(-(1 << kFixBits), -(1 << kFixBits), -(1 << kFixBits), 0);
            else reinterpret_cast<D4 *>(stage)[e] = D4{-1e30, -1e30, -1e30, 0.0};
        }
        __syncthreads();
        for (int slot = warp; slot < cnt; slot += nwarp) {
            // the home bead-atom: its own cell, image 0
            const E4 hp = reinterpret_cast<const E4 *>(d.cpos)[(size_t)cell * d.cap + slot];
            const int gi = d.cidx[(size_t)cell * d.cap + slot];
            unsigned *row = d.nbr + (size_t)gi * maxnb;
            int n = scount[slot];
            auto test = [&](const E4 &pj) {
                R dx, dy, dz;
                if (PM == PM_FIX) {
                    dx = (R)(int)((unsigned)pj.x - (unsigned)hp.x) * sx;
                    dy = (R)(int)((unsigned)pj.y - (unsigned)hp.y) * sy;
                    dz = (R)(int)((unsigned)pj.z - (unsigned)hp.z) * sz;
                } else {
                    dx = (R)(pj.x - hp.x) * lam;
                    dy = (R)(pj.y - hp.y) * lam;
                    dz = (R)(pj.z - hp.z) * lam;
                }
                const R r2 = fma(dx, dx, fma(dy, dy, dz * dz));
                // the home bead-atom itself (r2 == 0) and the sentinels fail
                const bool take = pass == 0 ? (r2 < rc2 && r2 > R(0)) : (r2 >= rc2 && r2 < rl2);
                const unsigned m = __ballot_sync(0xffffffffu, take);
                if (take) {
                    const int k = n + __popc(m & lt);
                    if (k < maxnb) row[k] = (unsigned)pj.w;
                }
                n += __popc(m);
            };
            for (int e0 = 0; e0 < padded; e0 += 64) {
                const E4 pa = stage[e0 + lane], pb = stage[e0 + 32 + lane];
                test(pa);
                test(pb);
            }
            if (lane == 0) scount[slot] = n;
        }
    }
    __syncthreads();
    for (int t = threadIdx.x; t < cnt; t += blockDim.x) {
        const int gi = d.cidx[(size_t)cell * d.cap + t];
        d.nnb[gi] = min(scount[t], maxnb);
        if (scount[t] > maxnb) atomicOr(d.err, (unsigned)ERR_NBR_OVERFLOW);
    }
}


// ---------------------------------------------------------------------------
// Pair force: Buckingham (energy-shifted) + damped shifted force Coulomb.

__device__ __forceinline__ float my_exp(float x) { return expf(x); }
__device__ __forceinline__ double my_exp(double x) { return exp(x); }
__device__ __forceinline__ float my_erfc(float x) { return erfcf(x); }
__device__ __forceinline__ double my_erfc(double x) { return erfc(x); }
__device__ __forceinline__ float my_sqrt(float x) { return sqrtf(x); }
__device__ __forceinline__ double my_sqrt(double x) { return sqrt(x); }

// Coefficients of one type pair, staged in shared memory by the step kernel
// (the pair type varies across the lanes of a warp).
template <class R> struct alignas(8 * sizeof(R)) PairRow {
    R inv_rho, A_over_rho, C6, qq, A, C, eshift, pad;
};

template <class R> __device__ __forceinline__ PairRow<R> pair_row(const PairTabT<R> &T, int t)
{
    PairRow<R> p;
    p.inv_rho = T.inv_rho[t]; p.A_over_rho = T.A_over_rho[t]; p.C6 = T.C6[t]; p.qq = T.qq[t];
    p.A = T.A[t]; p.C = T.C[t]; p.eshift = T.eshift[t]; p.pad = R(0);
    return p;
}

// -dV/dr / r and V of one pair at squared distance r2 < rc^2, FP32 form:
// branch-free, 1/r from rsqrt + one Newton step, the steep Buckingham
// exponential by expf (its argument reaches ~50), exp(-alpha^2 r^2) (argument
// < 3) through exp2, erfc(x) = exp(-x^2) P(u) with the fitted polynomial of the
// table.  This file is compiled without automatic multiply-add contraction:
// every fused multiply-add is written out, so that all kernels round alike.
__device__ __forceinline__ void pair_eval(const PairTabT<float> &T, const PairRow<float> &P2, float r2, float &f_over_r,
                                          float &e, bool energy = true)
{
    float rinv = rsqrtf(r2);
    rinv = rinv * fmaf(-0.5f * r2, rinv * rinv, 1.5f);
    const float r = r2 * rinv;
    const float r2i = rinv * rinv;
    const float r6i = r2i * r2i * r2i;
    const float ex = expf(-r * P2.inv_rho);                  // exp(-r/rho); A = 0 rows give 0 below
    const float gg = exp2f(-T.alpha2_l2e * r2);              // exp(-alpha^2 r^2)
    const float u = fmaf(T.alpha * r, T.erfc_us, -1.0f);
    float P = T.erfc_c[11];
#pragma unroll
    for (int k = 10; k >= 0; --k) P = fmaf(P, u, T.erfc_c[k]);
    const float er = gg * P;                                  // erfc(alpha r)
    const float qq = P2.qq;
    // A/rho e^{-r/rho} - 6C/r^7 + qq (erfc/r^2 + 2a/sqrt(pi) e^{-a^2 r^2}/r - fshift), times 1/r
    const float fb = fmaf(P2.A_over_rho, ex, -(P2.C6 * r6i * rinv));
    const float fc = fmaf(er, r2i, fmaf(T.two_a_sqrtpi * gg, rinv, -T.fshift));
    f_over_r = fmaf(qq, fc, fb) * rinv;
    if (energy) {
        const float ec = fmaf(er, rinv, fmaf(T.fshift, r - T.rc, -T.erfc_rc_over_rc));
        e = fmaf(qq, ec, fmaf(P2.A, ex, fmaf(-P2.C, r6i, -P2.eshift)));
    } else {
        e = 0.0f;
    }
}

// FP64 form: library exp / erfc / sqrt (the reference-accuracy path)
template <class R>
__device__ __forceinline__ void pair_eval(const PairTabT<R> &T, const PairRow<R> &P2, R r2, R &f_over_r, R &e,
                                          bool energy = true)
{
    const R r = my_sqrt(r2);
    const R rinv = R(1) / r;
    R f = 0, en = 0;
    const R A = P2.A, Cc = P2.C;
    if (A != R(0)) {
        const R ex = my_exp(-r * P2.inv_rho);
        f = P2.A_over_rho * ex;
        en = A * ex;
    }
    if (Cc != R(0)) {
        const R r2i = rinv * rinv;
        const R r6i = r2i * r2i * r2i;
        f = fma(-P2.C6 * r6i, rinv, f);
        en = fma(-Cc, r6i, en);
    }
    en -= P2.eshift;
    const R qq = P2.qq;
    if (qq != R(0)) {
        const R er = my_erfc(T.alpha * r);
        const R gg = my_exp(-T.alpha2 * r2);
        f = fma(qq, fma(er * rinv, rinv, fma(T.two_a_sqrtpi * gg, rinv, -T.fshift)), f);
        if (energy) en = fma(qq, fma(er, rinv, fma(T.fshift, r - T.rc, -T.erfc_rc_over_rc)), en);
    }
    f_over_r = f * rinv;
    e = en;
}

// Per-system reduction of the partials part[c0..c1) into the observable record
// (fixed summation order).  Executed by one CTA; sh holds one row per warp.
// FFP: the partials are float-float (hi, lo) pairs (FP32 list force kernel),
// summed on the FP32 pipe; otherwise FP64.  The record's entries are then
// formed in FP64, one per thread.
template <bool FFP>
static __device__ void reduce_system(const Dev &d, int s, long long step, int record, double (*sh)[kNQ + 1],
                                     const double *part, int c0, int c1)
{
    __shared__ double tot[kNQ + 1];
    const DSys S = d.sys[s];
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31, nw = blockDim.x >> 5;
    // the integrators' spring partials (ring polymers only: zero for one bead)
    double sp = 0.0;
    if (S.P > 1)
        for (int c = S.icta0 + (int)threadIdx.x; c < S.icta1; c += blockDim.x) sp += d.ipart[(size_t)c * kNQ + Q_SPRING];
    if (S.P > 1) sp = warp_sum(sp);
    if constexpr (FFP) {
        const float2 *P2 = reinterpret_cast<const float2 *>(part);
        FF acc[kNQ];
#pragma unroll
        for (int q = 0; q < kNQ; ++q) acc[q] = FF{0.f, 0.f};
        for (int c = c0 + (int)threadIdx.x; c < c1; c += blockDim.x)
#pragma unroll
            for (int q = 0; q < kNQ; ++q) {
                const float2 v = P2[(size_t)c * kNQ + q];
                acc[q].add_ff(v.x, v.y);
            }
        float2 (*sf)[kNQ + 1] = reinterpret_cast<float2 (*)[kNQ + 1]>(sh);
#pragma unroll
        for (int q = 0; q < kNQ; ++q) {
            acc[q].warp_reduce();
            if (lane == 0) sf[warp][q] = make_float2(acc[q].hi, acc[q].lo);
        }
        if (lane == 0) sh[warp][kNQ] = sp;  // the row's last entry (sf[warp][q] overlays sh[warp][q])
        __syncthreads();
        if (threadIdx.x < kNQ) {
            FF t{0.f, 0.f};
            for (int w = 0; w < nw; ++w) t.add_ff(sf[w][threadIdx.x].x, sf[w][threadIdx.x].y);
            tot[threadIdx.x] = (double)t.hi + (double)t.lo;
        } else if (threadIdx.x == kNQ) {
            double t = 0.0;
            for (int w = 0; w < nw; ++w) t += sh[w][kNQ];
            tot[kNQ] = t;
        }
    } else {
        double acc[kNQ];
        for (int q = 0; q < kNQ; ++q) acc[q] = 0.0;
        for (int c = c0 + (int)threadIdx.x; c < c1; c += blockDim.x)
            for (int q = 0; q < kNQ; ++q) acc[q] += part[(size_t)c * kNQ + q];
        for (int q = 0; q < kNQ; ++q) acc[q] = warp_sum(acc[q]);
        if (lane == 0) {
            for (int q = 0; q < kNQ; ++q) sh[warp][q] = acc[q];
            sh[warp][kNQ] = sp;
        }
        __syncthreads();
        if (threadIdx.x <= kNQ) {
            double t = 0.0;
            for (int w = 0; w < nw; ++w) t += sh[w][threadIdx.x];
            tot[threadIdx.x] = t;
        }
    }
    __syncthreads();
    const int q = threadIdx.x;
    if (q < QTB_NREC) {
        const double invP = S.invP;
        const double K = tot[Q_K], V = tot[Q_V] * invP, spr = tot[kNQ];
        double r = 0.0;
        if (q == 0) r = (double)step;
        else if (q == 1) r = K;
        else if (q == 2) r = V;
        else if (q == 3) r = spr;
        else if (q == 4) r = K - spr + V;
        else if (q < 14) {
            const int a = q - 5;  // xx xy xz / yx yy yz / zx zy zz
            const int m = (a == 0) ? 0 : (a == 4) ? 1 : (a == 8) ? 2 : (a == 1 || a == 3) ? 3 : (a == 2 || a == 6) ? 4 : 5;
            r = tot[Q_VIR + m] * invP;
        } else if (q < 17) r = tot[Q_MOM + q - 14];
        else if (q == 17) r = tot[Q_X2] * invP;
        else if (q == 20) {  // cell volume: the reference cell scaled by lam^3 in an isothermal-isobaric run
            const double l = (d.npt && d.npt[s].on) ? d.npt[s].lam : 1.0;
            r = S.box[0] * S.box[1] * S.box[2] * l * l * l;
        } else if (S.P == 1) {
            // centroid-virial estimators: for one bead 3N k_B T/2 and K, the
            // centroid kinetic energy K and virial trace; ring polymers get them
            // from the centroid kernel that follows
            if (q == 18) r = 1.5 * S.N * kBoltz * S.T;
            else if (q == 19 || q == 21) r = K;
            else r = (tot[Q_VIR + 0] * invP + tot[Q_VIR + 1] * invP) + tot[Q_VIR + 2] * invP;  // q == 22
        }
        if (q == 0 && (!isfinite(K) || !isfinite(V))) atomicOr(d.err, (unsigned)ERR_NONFINITE);
        d.latest[(size_t)s * QTB_NREC + q] = r;
        if (record >= 0 && step % d.obs_stride == 0) {
            const long long rr = step / d.obs_stride - 1;
            const int slot = (int)(rr % d.max_records);
            d.series[((size_t)slot * d.nsys + s) * QTB_NREC + q] = r;
        }
    }
}

// Isothermal-isobaric cells (Sec. 2.1, refs [11, 12]; the equations are those of
// qtb_params::npt): the update of system s's cell at the start of absolute step
// n (step j = n mod 256 of its block, positions in pos[cur], cur = j & 1), by one
// thread, from the kinetic energy and virial that the previous step's force
// launch reduced into the latest record:
//   B_e(dt/2) (the previous step's closing half, when due) and B_e(dt/2):
//       p_e += dt/2 (2 alpha K + W_vir - 3 V P_ext), twice;
//   the particles' first B(dt/2) factors for v_e = p_e / W: e1 = exp(-x),
//       g1 = (1 - e^{-x})/x, x = alpha v_e dt/2;
//   A(dt/2): lam <- lam e^{y}, y = v_e dt/2; the particles' drift in the
//       reference cell a1 = dt/2 (e^y - 1)/y / lam_new;
//   O(dt) of the cell: p_e <- ce p_e + sqrt((1 - ce^2) W k_B T) xi,
//       xi from Philox stream 1, dof 0, step n;
//   A(dt/2) with the new v_e (a2, lam), and the closing B(dt/2) factors e2, g2.
// A list rebuild is requested for this step's force launch when the cell scale
// has moved by more than kNptCellSkin skin over the list radius since the system's last
// rebuild; a cell below kCellMinScale raises ERR_CELL.
// FP32 form: the transcendental factors in FP32 (this GPU's FP64 rate is a small
// fraction of its FP32 rate and the kernel is one thread's dependent chain); the
// cell momentum, G and lam stay FP64, lam advanced as lam + lam (e^y - 1).
__device__ __forceinline__ double xm1_over_x(double x) { return x != 0.0 ? expm1(x) / x : 1.0; }
__device__ __forceinline__ float xm1_over_xf(float x)
{
    // (e^x - 1)/x: Taylor to x^3 near 0 (the next term is below 1e-14 for |x| < 1e-3)
    return fabsf(x) < 1e-3f ? fmaf(x, fmaf(x, fmaf(x, 1.0f / 24.0f, 1.0f / 6.0f), 0.5f), 1.0f) : expm1f(x) / x;
}

template <bool F32>
__device__ void cell_update(const Dev &d, int s, long long n, int cur)
{
    DNpt C = d.npt[s];
    const DSys &S = d.sys[s];
    const double *rec = d.latest + (size_t)s * QTB_NREC;
    const double K = rec[21], Wv = rec[22];  // centroid kinetic energy and virial (one bead: K, W)
    const double V = S.box[0] * S.box[1] * S.box[2] * C.lam * C.lam * C.lam;
    const double G = 2.0 * C.alpha * K + Wv - 3.0 * V * C.pext;
    const double h = 0.5 * d.dt;
    if (C.pending) C.peps += h * G;
    C.peps += h * G;
    // the cell's random force: Philox stream 1, dof 0, step n
    const long long q = (n >= 0) ? n / 4 : -((-n + 3) / 4);
    const unsigned long long uq = (unsigned long long)q;
    const uint4 w = philox4x32_10(make_uint4((uint32_t)uq, 0u, 1u, (uint32_t)(uq >> 32)), (uint32_t)d.seed,
                                  (uint32_t)(d.seed >> 32) ^ (uint32_t)s);
    const int e = (int)(n - 4 * q);
    const uint32_t wa = (e < 2) ? w.x : w.z, wb = (e < 2) ? w.y : w.w;
    double lam;
    if constexpr (F32) {
        const float hf = (float)h, af = (float)C.alpha;
        float ve = (float)C.peps * C.inv_wf;
        float x = af * ve * hf, y = ve * hf;
        C.e1f = expf(-x);
        C.g1f = xm1_over_xf(-x);
        lam = fma(C.lam, (double)expm1f(y), C.lam);
        C.a1f = hf * xm1_over_xf(y) / (float)lam;
        const float u1 = ((float)wa + 1.0f) * 2.3283064365386963e-10f, u2 = (float)wb * 2.3283064365386963e-10f;
        float sn, cs;
        sincospif(2.0f * u2, &sn, &cs);
        const float xi = sqrtf(-2.0f * logf(u1)) * ((e & 1) ? sn : cs);
        C.peps = fma(C.ce, C.peps, C.sige * (double)xi);
        ve = (float)C.peps * C.inv_wf;
        x = af * ve * hf;
        y = ve * hf;
        lam = fma(lam, (double)expm1f(y), lam);
        C.a2f = hf * xm1_over_xf(y) / (float)lam;
        C.e2f = expf(-x);
        C.g2f = xm1_over_xf(-x);
        C.lamf = (float)lam;  // (the FP32 kernels read only the float coefficients)
    } else {
        double ve = C.peps / C.W;
        double x = C.alpha * ve * h;
        C.e1 = exp(-x);
        C.g1 = xm1_over_x(-x);
        double y = ve * h;
        lam = C.lam * exp(y);
        C.a1 = h * xm1_over_x(y) / lam;
        const double u1 = ((double)wa + 1.0) * 2.3283064365386963e-10, u2 = (double)wb * 2.3283064365386963e-10;
        double sn, cs;
        sincospi(2.0 * u2, &sn, &cs);
        const double xi = sqrt(-2.0 * log(u1)) * ((e & 1) ? sn : cs);
        C.peps = C.ce * C.peps + C.sige * xi;
        ve = C.peps / C.W;
        y = ve * h;
        lam = lam * exp(y);
        C.a2 = h * xm1_over_x(y) / lam;
        x = C.alpha * ve * h;
        C.e2 = exp(-x);
        C.g2 = xm1_over_x(-x);
        C.e1f = (float)C.e1; C.g1f = (float)C.g1; C.a1f = (float)C.a1; C.a2f = (float)C.a2;
        C.e2f = (float)C.e2; C.g2f = (float)C.g2; C.lamf = (float)lam;
    }
    // ring polymers: the bead offsets keep their physical length across the update
    if constexpr (F32) {
        C.lam_oldf = (float)C.lam;
        C.inv_lamf = 1.0f / (float)lam;
    } else {
        C.lam_old = C.lam;
        C.inv_lam = 1.0 / lam;
    }
    C.lam = lam;
    C.pending = 1;
    d.npt[s] = C;
    if (!(lam >= kCellMinScale) || !isfinite(lam)) atomicOr(d.err, (unsigned)ERR_CELL);
    if (fabs(lam - C.lam_rb) > C.rb_tol * C.lam_rb) {
        atomicOr(&d.rflag[cur * d.nsys + s], 1u);
        atomicOr(&d.flag[cur], 1u);
    }
}

// ---------------------------------------------------------------------------
// Pair force from the neighbour lists: LPA lanes per home bead-atom
// (32 / LPA bead-atoms per warp), each lane strides through the list with two
// independent entries per iteration and the next iteration's entries already
// requested; every entry is evaluated and masked by r < r_cut (no divergent
// branch).  Epilogue on the first three lanes of a group (one Cartesian
// component each): force (times 1/P, Eq. 4), the closing B(dt/2) kick, the
// observables of recorded steps and, with ADV (one-bead systems), the first
// half of the next step: B(dt/2), A(dt/2) O(dt) A(dt/2) with the next step's
// coloured noise, written to x and pos[cur ^ 1], and the rebuild test for the
// next step.  Recorded steps: the last CTA of a system reduces its partials.

template <int PM, class R, int ADV, int REC, int LPA, int MI>
__device__ __forceinline__ void force_unit(const Dev &d, const PairTabT<R> &T, const PairRow<R> *ptab, int kick,
                                           int j, int cur, int u, double (*red)[kNQ], double (*rsh)[kNQ + 1],
                                           int &s_last)
{
    typedef typename std::conditional<PM == PM_FIX, int4, D4>::type E4;
    typedef typename std::conditional<sizeof(R) == 4, FF, DD>::type ACC;
    typedef typename PosT<PM, R>::S PS;
    constexpr int APW = 32 / LPA;
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int sub = lane & (LPA - 1), grp = lane / LPA;
    const DRep RP = d.rep[d.lcta_rep[u]];
    const int i = (u - RP.fcta0) * list_atoms(LPA) + warp * APW + grp;
    const bool act = i < RP.N;
    const long long step = d.clock[0] * kBlockSteps + j + 1;
    // (isothermal-isobaric runs reduce K and the virial every step: the cell needs them)
    const bool rec = REC && ((kick == 0) || (step % d.obs_stride == 0) || d.npt != nullptr);
    const DSys &S = d.sys[RP.sys];
    const size_t G = (size_t)d.G;
    const long long gi = RP.g0 + (act ? i : 0);
    const E4 *Pc = reinterpret_cast<const E4 *>(d.pos[cur]);
    const E4 *Pr = Pc + RP.g0;
    const E4 hp = Pc[gi];
    int ti;
    if (PM == PM_FIX) ti = hp.w; else ti = (int)hp.w;
    const int n = act ? min(d.nnb[gi], d.maxnb) : 0;
    const unsigned *row = d.nbr + (size_t)gi * d.maxnb;
    // physical distances: the reference cell's, scaled by lam in an isothermal-isobaric run
    // (such runs launch the recording variants only: the others carry no cell code)
    const DNpt *NC = (REC && d.npt && d.npt[RP.sys].on) ? d.npt + RP.sys : nullptr;
    const R lam = NC ? (sizeof(R) == 4 ? (R)NC->lamf : (R)NC->lam) : R(1);
    const R sx = (R)RP.fix_scale[0] * lam, sy = (R)RP.fix_scale[1] * lam, sz = (R)RP.fix_scale[2] * lam;
    const R rc2 = T.rc2;
    ACC fx{}, fy{}, fz{};
    R en = 0, w0 = 0, w1 = 0, w2 = 0, w3 = 0, w4 = 0, w5 = 0;
    struct Geo {
        R dx, dy, dz, r2;
        int tj;
    };
    // r_j + image - r_i of one list entry
    auto geo = [&](unsigned e) {
        const E4 pj = Pr[e & kNbIdx];
        Geo g;
        if (PM == PM_FIX) {
            // exact in wrapping 32-bit arithmetic
            if constexpr (MI) {
                // MI: every cell exceeds twice the largest separation a list entry can
                // reach, so the difference modulo the 30-bit edge, sign-extended, is the
                // entry's image (4 x the difference, exact in float, times scale/4: the
                // same value as below, without decoding the image bits)
                g.dx = (R)(int)(((unsigned)pj.x - (unsigned)hp.x) << 2) * (sx * R(0.25));
                g.dy = (R)(int)(((unsigned)pj.y - (unsigned)hp.y) << 2) * (sy * R(0.25));
                g.dz = (R)(int)(((unsigned)pj.z - (unsigned)hp.z) << 2) * (sz * R(0.25));
            } else {
                g.dx = (R)(int)((unsigned)pj.x + ((e << 4) & 0xC0000000u) - (unsigned)hp.x) * sx;
                g.dy = (R)(int)((unsigned)pj.y + ((e << 2) & 0xC0000000u) - (unsigned)hp.y) * sy;
                g.dz = (R)(int)((unsigned)pj.z + (e & 0xC0000000u) - (unsigned)hp.z) * sz;
            }
            g.tj = pj.w;
        } else {
            // image from m mod 4: code 2 is +2 or -2, told apart by the sign of
            // the raw difference (the box exceeds r_cut/2 + skin)
            const double pd[3] = {(double)pj.x - (double)hp.x, (double)pj.y - (double)hp.y, (double)pj.z - (double)hp.z};
            R dv[3];
#pragma unroll
            for (int c = 0; c < 3; ++c) {
                const int code = (int)((e >> (26 + 2 * c)) & 3u);
                const int m = (code == 3) ? -1 : (code == 2) ? (pd[c] > 0.0 ? -2 : 2) : code;
                dv[c] = (R)(pd[c] + m * RP.box[c]) * lam;
            }
            g.dx = dv[0]; g.dy = dv[1]; g.dz = dv[2];
            g.tj = (int)pj.w;
        }
        g.r2 = fma(g.dx, g.dx, fma(g.dy, g.dy, g.dz * g.dz));
        return g;
    };
    // force (and on recorded steps energy and virial) of one entry, masked by `in`,
    // added to the round's partial sums (px, py, pz)
    auto force = [&](const Geo &g, bool in, R &px, R &py, R &pz) {
        R fo, ee;
        pair_eval(T, ptab[ti * kMaxTypes + g.tj], g.r2, fo, ee, REC && rec);
        fo = in ? fo : R(0);
        // stored displacement is r_j - r_i: the force on i is -fo (r_j - r_i)
        px = fma(-fo, g.dx, px); py = fma(-fo, g.dy, py); pz = fma(-fo, g.dz, pz);
        if (REC && rec) {
            en += in ? ee : R(0);
            w0 = fma(fo * g.dx, g.dx, w0); w1 = fma(fo * g.dy, g.dy, w1); w2 = fma(fo * g.dz, g.dz, w2);
            w3 = fma(fo * g.dx, g.dy, w3); w4 = fma(fo * g.dx, g.dz, w4); w5 = fma(fo * g.dy, g.dz, w5);
        }
    };
    {
        // entries k + q LPA (q < NE) of this lane; the next NE are requested before
        // the current ones are evaluated (slots past the end read entry 0, masked).
        // The lists end with the skin-shell entries: a round in which no lane of
        // the warp has an entry within r_cut skips the pair terms (they would add
        // exact zeros).  The trip count is the warp's longest list, so the vote
        // is uniform.
        constexpr int NE = 4;
        int nmax = n;
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) nmax = max(nmax, __shfl_xor_sync(0xffffffffu, nmax, o));
        unsigned e[NE];
#pragma unroll
        for (int q = 0; q < NE; ++q) e[q] = (sub + q * LPA < n) ? row[sub + q * LPA] : 0u;
        for (int k0 = 0; k0 < nmax; k0 += NE * LPA) {
            const int k = k0 + sub, kn = k + NE * LPA;
            unsigned e2[NE];
#pragma unroll
            for (int q = 0; q < NE; ++q) e2[q] = (kn + q * LPA < n) ? row[kn + q * LPA] : 0u;
            Geo g[NE];
            bool in[NE], any = false;
#pragma unroll
            for (int q = 0; q < NE; ++q) {
                g[q] = geo(e[q]);
                in[q] = (k + q * LPA < n) && (g[q].r2 < rc2);
                any |= in[q];
            }
            if (__any_sync(0xffffffffu, any)) {
                // the round's NE terms are summed in R, the partial sum then added
                // error-free (float-float): the extra roundings are those of NE - 1
                // additions of terms of like size (modelled on the CPU: no change of
                // the error budget)
                R px = 0, py = 0, pz = 0;
#pragma unroll
                for (int q = 0; q < NE; ++q) force(g[q], in[q], px, py, pz);
                fx.add(px); fy.add(py); fz.add(pz);
            }
#pragma unroll
            for (int q = 0; q < NE; ++q) e[q] = e2[q];
        }
    }
    fx.template group_reduce<LPA>(); fy.template group_reduce<LPA>(); fz.template group_reduce<LPA>();
    // recorded steps: the FP64 form sums its partials in FP64; the FP32 form in
    // float-float on the FP32 pipe (this GPU's FP64 rate is a small fraction of
    // its FP32 rate), kc and mc being a component lane's kinetic energy and momentum
    constexpr bool kFF = sizeof(R) == 4;
    double acc[kNQ];
#pragma unroll
    for (int q = 0; q < kNQ; ++q) acc[q] = 0.0;
    float kc = 0.f, kl = 0.f, mc = 0.f, ml = 0.f;  // float-float (hi, lo)
    if (REC && rec) {
        en = group_sum<LPA>(en);
        w0 = group_sum<LPA>(w0); w1 = group_sum<LPA>(w1); w2 = group_sum<LPA>(w2);
        w3 = group_sum<LPA>(w3); w4 = group_sum<LPA>(w4); w5 = group_sum<LPA>(w5);
        if (!kFF && act && sub == 0) {
            acc[Q_V] = 0.5 * (double)en;
            acc[Q_VIR + 0] = 0.5 * (double)w0; acc[Q_VIR + 1] = 0.5 * (double)w1;
            acc[Q_VIR + 2] = 0.5 * (double)w2; acc[Q_VIR + 3] = 0.5 * (double)w3;
            acc[Q_VIR + 4] = 0.5 * (double)w4; acc[Q_VIR + 5] = 0.5 * (double)w5;
        }
    }
    R dd = 0;  // squared displacement component since the last rebuild (ADV)
    if (act && sub < 3) {
        const int c = sub;
        const R invP = sizeof(R) == 4 ? (R)S.invP_f : (R)S.invP;
        const R fc = (R)(c == 0 ? fx.value() : c == 1 ? fy.value() : fz.value()) * invP;
        R *Fo = reinterpret_cast<R *>(d.f);
        R *V = reinterpret_cast<R *>(d.v);
        const size_t o = (size_t)c * G + gi;
        Fo[o] = fc;
        const R hdtm = T.hdt_m[ti];
        R v = V[o];
        if (kick) {
            if (NC && S.P == 1) {  // B(dt/2) with the cell's friction: v e2 + (hdt/m) F g2
                // (ring polymers: the plain kick here, the centroid's friction in k_centroid)
                const R e2 = sizeof(R) == 4 ? (R)NC->e2f : (R)NC->e2, g2 = sizeof(R) == 4 ? (R)NC->g2f : (R)NC->g2;
                v = fma(v, e2, (hdtm * fc) * g2);
            } else {
                v = fma(hdtm, fc, v);
            }
        }
        if (REC && rec) {
            if constexpr (kFF) {
                // m v^2 / 2 and m v to ~1e-14: v^2 = p + pe exactly, the masses float-float
                const float vf = (float)v, p = vf * vf, pe = fmaf(vf, vf, -p);
                const float2 hm = T.half_mvv_ff[ti], mm = T.mass_ff[ti];
                kc = hm.x * p;
                kl = fmaf(hm.x, p, -kc) + fmaf(hm.x, pe, hm.y * p);
                mc = mm.x * vf;
                ml = fmaf(mm.x, vf, -mc) + mm.y * vf;
            } else {
                acc[Q_K] += 0.5 * T.mass_mvv[ti] * (double)v * (double)v;
                acc[Q_MOM + c] += T.mass[ti] * (double)v;
            }
        }
        if (ADV && !NC) {
            // next step, one bead (the mode is the bead): B(dt/2), A(dt/2) O(dt) A(dt/2)
            // (with a cell, after the cell's update: npt_next_half)
            const R *rot = reinterpret_cast<const R *>(d.rot) + 3 * S.rot0;
            const R cs = rot[0], sw = rot[1], ws = rot[2];
            const R sig = reinterpret_cast<const R *>(d.osig)[RP.sys * kMaxTypes + ti];
            const R c1 = sizeof(R) == 4 ? (R)S.c1_f : (R)S.c1;
            const R eta = reinterpret_cast<const R *>(d.eta)[eta_row(d, j + 1) * d.Dtot + S.dof0 + (size_t)c * S.N + i];
            R pk = fma(hdtm, fc, v);
            R qq = 0;
            mode_aoa(qq, pk, cs, sw, ws, c1, sig * eta);
            v = pk;
            PS *X = reinterpret_cast<PS *>(d.x);
            const float fsc = S.fix_scale[c];
            const PS xn = PosT<PM, R>::add(X[o], qq, S.box[c], fsc, S.fix_inv[c]);
            X[o] = xn;
            reinterpret_cast<PS *>(d.pos[cur ^ 1])[4 * (size_t)gi + c] = xn;
            const R dc = PosT<PM, R>::diff(xn, reinterpret_cast<const PS *>(d.xref)[o], fsc);
            dd = dc * dc;
        }
        if (kick || ADV) V[o] = v;
    }
    if (ADV) {
        const int b0 = grp * LPA;
        const R tot = __shfl_sync(0xffffffffu, dd, b0) + __shfl_sync(0xffffffffu, dd, b0 + 1) +
                      __shfl_sync(0xffffffffu, dd, b0 + 2);
        const R lim = sizeof(R) == 4 ? (R)S.skin2_f : (R)S.skin2;
        if (__any_sync(0xffffffffu, act && sub == 0 && tot > lim) && lane == 0) {
            atomicOr(&d.rflag[(cur ^ 1) * d.nsys + RP.sys], 1u);
            atomicOr(&d.flag[cur ^ 1], 1u);
        }
    }
    if (REC && rec) {
        if constexpr (kFF) {
            cta_store_partials_ff<LPA>(act && sub == 0, en, w0, w1, w2, w3, w4, w5, kc, kl, mc, ml, red,
                                       reinterpret_cast<float2 *>(d.part) + (size_t)u * kNQ);
        } else {
#pragma unroll
            for (int q = 0; q < kNQ; ++q) acc[q] = warp_sum(acc[q]);
            cta_store_partials(acc, red, d.part + (size_t)u * kNQ);
        }
        // two levels, in fixed groups of kRedGroup consecutive units of the system:
        // the CTA that finishes a group's last unit sums the group's partials (unit
        // order), the one that finishes the system's last group forms the record
        // from the group sums (group order); partials made visible first.  The
        // order depends on the system's units only, so a system of a batch reduces
        // as it would alone.
        __threadfence();
        __syncthreads();
        const int g = (u - S.fcta0) / kRedGroup, gu0 = S.fcta0 + g * kRedGroup;
        const int gn = min(kRedGroup, S.fcta1 - gu0);
        if (threadIdx.x == 0) {
            const unsigned prev = atomicAdd(&d.gdone[S.grp0 + g], 1u);
            s_last = (prev == (unsigned)(gn - 1)) ? 1 : 0;
        }
        __syncthreads();
        if (s_last) {
            __threadfence();
            if (threadIdx.x < kNQ) {
                const int q = threadIdx.x;
                if constexpr (kFF) {
                    const float2 *P2 = reinterpret_cast<const float2 *>(d.part);
                    float2 v[kRedGroup];
#pragma unroll
                    for (int k = 0; k < kRedGroup; ++k)
                        v[k] = (k < gn) ? __ldcg(P2 + (size_t)(gu0 + k) * kNQ + q) : make_float2(0.f, 0.f);
                    FF t{0.f, 0.f};
#pragma unroll
                    for (int k = 0; k < kRedGroup; ++k) t.add_ff(v[k].x, v[k].y);
                    reinterpret_cast<float2 *>(d.gpart)[(size_t)(S.grp0 + g) * kNQ + q] = make_float2(t.hi, t.lo);
                } else {
                    double v[kRedGroup];
#pragma unroll
                    for (int k = 0; k < kRedGroup; ++k) v[k] = (k < gn) ? __ldcg(d.part + (size_t)(gu0 + k) * kNQ + q) : 0.0;
                    double t = 0.0;
#pragma unroll
                    for (int k = 0; k < kRedGroup; ++k) t += v[k];
                    d.gpart[(size_t)(S.grp0 + g) * kNQ + q] = t;
                }
            }
            if (threadIdx.x == 0) d.gdone[S.grp0 + g] = 0u;
            __threadfence();
            __syncthreads();
            if (threadIdx.x == 0) {
                const unsigned prev = atomicAdd(&d.done[RP.sys], 1u);
                s_last = (prev == (unsigned)(S.ngrp - 1)) ? 1 : 0;
            }
            __syncthreads();
            if (s_last) {
                __threadfence();
                reduce_system<kFF>(d, RP.sys, step, kick ? 1 : -1, rsh, d.gpart, S.grp0, S.grp0 + S.ngrp);
                if (threadIdx.x == 0) d.done[RP.sys] = 0u;
                if (ADV && NC && kick) {
                    // the cell's update for the next step, from the record just formed
                    __syncthreads();
                    if (threadIdx.x == 0) cell_update<kFF>(d, RP.sys, step, cur ^ 1);
                }
            }
        }
    }
}

// Isothermal-isobaric runs (one bead per atom), fused steps: the first half of
// the next step, B(dt/2) A(dt/2) O(dt) A(dt/2) with the coefficients of the
// cell's update, for the bead-atoms of this CTA's force units, after the grid
// barrier that follows that update.  The arithmetic is the one-bead cell branch
// of k_integrate's, operation for operation, so that a fused step gives the
// same bits as an integrator launch would.  j1 is the next step (its noise row),
// nxt its position buffer.
template <int PM, class R, int LPA>
__device__ void npt_next_half(const Dev &d, int j1, int nxt)
{
    typedef typename PosT<PM, R>::S PS;
    constexpr int NA = list_atoms(LPA);
    __shared__ R sdd[3 * NA];
    const size_t G = (size_t)d.G;
    for (int u = blockIdx.x; u < d.nunits; u += gridDim.x) {
        const DRep RP = d.rep[d.lcta_rep[u]];
        const int s = RP.sys;
        const DSys &S = d.sys[s];
        const DNpt *NC = d.npt + s;
        const int t = threadIdx.x, k = t / 3, c = t - 3 * k;
        const int i = (u - RP.fcta0) * NA + k;
        const bool act = t < 3 * NA && i < RP.N;
        R dd = 0;
        if (act) {
            const size_t gi = RP.g0 + i, o = (size_t)c * G + gi;
            R *V = reinterpret_cast<R *>(d.v);
            const R *F = reinterpret_cast<const R *>(d.f);
            PS *X = reinterpret_cast<PS *>(d.x);
            const int ty = d.typ[S.g0 + i];
            const R hdtm = reinterpret_cast<const R *>(d.hdt_m)[ty];
            const R sig = reinterpret_cast<const R *>(d.osig)[s * kMaxTypes + ty];
            const R c1 = sizeof(R) == 4 ? (R)S.c1_f : (R)S.c1;
            const R e1 = sizeof(R) == 4 ? (R)NC->e1f : (R)NC->e1, g1 = sizeof(R) == 4 ? (R)NC->g1f : (R)NC->g1;
            const R a1 = sizeof(R) == 4 ? (R)NC->a1f : (R)NC->a1, a2 = sizeof(R) == 4 ? (R)NC->a2f : (R)NC->a2;
            const R eta = reinterpret_cast<const R *>(d.eta)[eta_row(d, j1) * d.Dtot + S.dof0 + (size_t)c * S.N + i];
            R pk = fma(V[o], e1, (hdtm * F[o]) * g1);
            R disp = pk * a1;
            pk = fma(c1, pk, sig * eta);
            disp = fma(pk, a2, disp);
            V[o] = pk;
            const float fsc = S.fix_scale[c];
            const PS xn = PosT<PM, R>::add(X[o], disp, S.box[c], fsc, S.fix_inv[c]);
            X[o] = xn;
            reinterpret_cast<PS *>(d.pos[nxt])[4 * gi + c] = xn;
            const R dc = PosT<PM, R>::diff(xn, reinterpret_cast<const PS *>(d.xref)[o], fsc);
            dd = dc * dc;
        }
        if (t < 3 * NA) sdd[t] = dd;
        __syncthreads();
        // the physical displacement (lam times the reference one) against D^2 (DSys::npt_d2)
        bool moved = false;
        if (act && c == 0) {
            const R tot = sdd[t] + sdd[t + 1] + sdd[t + 2];
            const R l = sizeof(R) == 4 ? (R)NC->lamf : (R)NC->lam;
            const R lim = (sizeof(R) == 4 ? (R)S.npt_d2_f : (R)S.npt_d2) / (l * l);
            moved = tot > lim;
        }
        if (__syncthreads_or(moved) && threadIdx.x == 0) {
            atomicOr(&d.rflag[nxt * d.nsys + s], 1u);
            atomicOr(&d.flag[nxt], 1u);
        }
    }
}

// One step of the pair-potential systems, a cooperative launch whose CTAs
// (at most one wave) loop over the force units (list_atoms(LPA) bead-atoms each).
// When the producer of this step's positions requested a rebuild (flag[cur]),
// the grid first bins, sorts and builds the lists, phases separated by grid
// barriers.  Dynamic shared memory: the staging chunk of the list build
// (stage_cap entries; also the sort keys).  FP32 form: at least 7 CTAs per SM
// (72 registers, no spills; 1064 resident CTAs hold the 1000 units of an
// 8000-ion crystal in one wave): 5 % faster there than 8 CTAs at 64 registers,
// no slower on larger systems; six or eight entries in flight per lane spill.
// The recording variants (energy and virial as well) take 4 CTAs per SM and
// spill nothing: 10 % faster per step on an isothermal-isobaric run, which
// records every step, and no slower on the 8000-ion crystal's recorded step.
template <int PM, class R, int ADV, int REC, int LPA, int MI>
__global__ void __launch_bounds__(32 * kListWarps, sizeof(R) == 4 ? (REC ? 4 : 7) : 4)
    k_step(Dev d, PairTabT<R> T, int kick, int j, int cur)
{
    extern __shared__ __align__(32) unsigned char fsm[];
    __shared__ BuildSmem B;
    __shared__ PairRow<R> ptab[kMaxTypes * kMaxTypes];
    if (threadIdx.x < kMaxTypes * kMaxTypes) ptab[threadIdx.x] = pair_row(T, threadIdx.x);
    __syncthreads();
    __shared__ double red[kListWarps][kNQ];
    __shared__ double rsh[kListWarps][kNQ + 1];
    __shared__ int s_last;
    wait_previous_step();
    // read by every thread before the flag can be cleared (after the first barrier)
    const bool rebuild = *(volatile const unsigned *)&d.flag[cur] != 0u;
    if (rebuild) {
        bin_phase<PM>(d, cur);
        grid_barrier(d);
        if (blockIdx.x == 0 && threadIdx.x == 0) {
            d.flag[cur] = 0u;  // this step's rebuild request is consumed
            atomicAdd(d.nrebuild, 1ull);
        }
        sort_phase<PM>(d, cur, reinterpret_cast<int *>(fsm));
        grid_barrier(d);
        for (int s = 0; s < d.nsys; ++s) {  // the cells of the requesting systems
            if (!d.rebuild_all && d.rflag[cur * d.nsys + s] == 0u) continue;  // uniform over the grid
            const int c0 = d.sys[s].cell0, c1 = d.sys[s].cell1, nb = (int)gridDim.x;
            for (int cell = c0 + (((int)blockIdx.x - c0) % nb + nb) % nb; cell < c1; cell += nb)
                build_cell<PM, R>(d, T.rc2, sizeof(R) == 4 ? (R)d.sys[s].rl2_f : (R)d.sys[s].rl2, cell, fsm, B);
        }
        grid_barrier(d);
        // the per-system requests were read by every phase: consumed now (their
        // next producer, of step s + 2, runs in a later launch); an isothermal-
        // isobaric cell remembers the scale its lists were built at
        if (blockIdx.x == 0)
            for (int t = threadIdx.x; t < d.nsys; t += blockDim.x) {
                if (d.npt && d.npt[t].on && (d.rebuild_all || d.rflag[cur * d.nsys + t] != 0u))
                    d.npt[t].lam_rb = d.npt[t].lam;
                d.rflag[cur * d.nsys + t] = 0u;
            }
    }
    release_next_step();
    for (int u = blockIdx.x; u < d.nunits; u += gridDim.x)
        force_unit<PM, R, ADV, REC, LPA, MI>(d, T, ptab, kick, j, cur, u, red, rsh, s_last);
    if constexpr (ADV && REC) {
        // isothermal-isobaric cells: the next step's first half waits for the
        // cells' updates (made by each system's last CTA) behind a grid barrier
        if (d.npt && kick) {
            grid_barrier(d);
            npt_next_half<PM, R, LPA>(d, j + 1, cur ^ 1);
        }
    }
}

template <int PM, class R, int ADV, int REC, int LPA, int MI>
static cudaError_t step_prepare_one(size_t smem, int nsm, int &grid)
{
    cudaError_t e = cudaFuncSetAttribute(k_step<PM, R, ADV, REC, LPA, MI>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    int per_sm = 0;
    e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_step<PM, R, ADV, REC, LPA, MI>, 32 * kListWarps, smem);
    grid = per_sm * nsm;
    return e;
}

template <int LPA>
static cudaError_t step_prepare_lanes(MdLaunch &m, int stage_entries)
{
    int dev = 0, nsm = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e == cudaSuccess) e = cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev);
    if (e != cudaSuccess) return e;
    m.step_smem = (size_t)stage_entries * (m.mixed ? sizeof(int4) : sizeof(D4));
    if (m.mixed && m.minimg) {
        if ((e = step_prepare_one<PM_FIX, float, 0, 0, LPA, 1>(m.step_smem, nsm, m.step_grid[0])) != cudaSuccess) return e;
        if ((e = step_prepare_one<PM_FIX, float, 0, 1, LPA, 1>(m.step_smem, nsm, m.step_grid[1])) != cudaSuccess) return e;
        if ((e = step_prepare_one<PM_FIX, float, 1, 0, LPA, 1>(m.step_smem, nsm, m.step_grid[2])) != cudaSuccess) return e;
        e = step_prepare_one<PM_FIX, float, 1, 1, LPA, 1>(m.step_smem, nsm, m.step_grid[3]);
    } else if (m.mixed) {
        if ((e = step_prepare_one<PM_FIX, float, 0, 0, LPA, 0>(m.step_smem, nsm, m.step_grid[0])) != cudaSuccess) return e;
        if ((e = step_prepare_one<PM_FIX, float, 0, 1, LPA, 0>(m.step_smem, nsm, m.step_grid[1])) != cudaSuccess) return e;
        if ((e = step_prepare_one<PM_FIX, float, 1, 0, LPA, 0>(m.step_smem, nsm, m.step_grid[2])) != cudaSuccess) return e;
        e = step_prepare_one<PM_FIX, float, 1, 1, LPA, 0>(m.step_smem, nsm, m.step_grid[3]);
    } else {
        if ((e = step_prepare_one<PM_BOX64, double, 0, 0, LPA, 0>(m.step_smem, nsm, m.step_grid[0])) != cudaSuccess) return e;
        if ((e = step_prepare_one<PM_BOX64, double, 0, 1, LPA, 0>(m.step_smem, nsm, m.step_grid[1])) != cudaSuccess) return e;
        if ((e = step_prepare_one<PM_BOX64, double, 1, 0, LPA, 0>(m.step_smem, nsm, m.step_grid[2])) != cudaSuccess) return e;
        e = step_prepare_one<PM_BOX64, double, 1, 1, LPA, 0>(m.step_smem, nsm, m.step_grid[3]);
    }
    return e;
}

// cooperative launch: all CTAs resident at once (the grid barriers need it)
template <int PM, class R, int ADV, int REC, int LPA, int MI>
static cudaError_t step_launch(const Dev &d, const MdLaunch &m, const PairTabT<R> &T, int kick, int j, int cur,
                               cudaStream_t st)
{
    const int grid = std::min(d.nunits, m.step_grid[ADV * 2 + REC]);
    if (grid < 1) return cudaErrorInvalidConfiguration;
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3((unsigned)grid);
    cfg.blockDim = dim3(32 * kListWarps);
    cfg.dynamicSmemBytes = m.step_smem;
    cfg.stream = st;
    cudaLaunchAttribute at[2];
    at[0].id = cudaLaunchAttributeCooperative;
    at[0].val.cooperative = 1;
    at[1].id = cudaLaunchAttributeProgrammaticStreamSerialization;  // see wait_previous_step
    at[1].val.programmaticStreamSerializationAllowed = 1;
    cfg.attrs = at;
    cfg.numAttrs = 2;
    return cudaLaunchKernelEx(&cfg, k_step<PM, R, ADV, REC, LPA, MI>, d, T, kick, j, cur);
}

template <int PM, class R, int LPA, int MI>
static cudaError_t step_any(const Dev &d, const MdLaunch &m, const PairTabT<R> &T, int kick, int j, int cur, int adv,
                            int rec, cudaStream_t st)
{
    if (adv && rec) return step_launch<PM, R, 1, 1, LPA, MI>(d, m, T, kick, j, cur, st);
    if (adv) return step_launch<PM, R, 1, 0, LPA, MI>(d, m, T, kick, j, cur, st);
    if (rec) return step_launch<PM, R, 0, 1, LPA, MI>(d, m, T, kick, j, cur, st);
    return step_launch<PM, R, 0, 0, LPA, MI>(d, m, T, kick, j, cur, st);
}

// the step kernel of one lane count (one translation unit per count)
template <int LPA>
static cudaError_t step_force_lanes(const Dev &d, const MdLaunch &m, const PairTabT<float> &Tf,
                                    const PairTabT<double> &Td, int kick, int j, int cur, int adv, int rec,
                                    cudaStream_t st)
{
    if (m.mixed && m.minimg) return step_any<PM_FIX, float, LPA, 1>(d, m, Tf, kick, j, cur, adv, rec, st);
    if (m.mixed) return step_any<PM_FIX, float, LPA, 0>(d, m, Tf, kick, j, cur, adv, rec, st);
    return step_any<PM_BOX64, double, LPA, 0>(d, m, Td, kick, j, cur, adv, rec, st);
}

}  // namespace qtb
