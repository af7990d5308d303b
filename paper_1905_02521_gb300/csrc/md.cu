// md.cu -- cell lists, pair and external forces, the normal-mode BAOAB
// integrator and the per-system reductions (sm_103a).
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

template <class R> struct PosT<PM_BOX64, R> {  // FP64, wrapped into [0, L)
    typedef double S;
    __device__ static R rel(S a, S b, double L, float, float)
    {
        double d = a - b;
        return (R)(d - L * rint(d / L));
    }
    __device__ static S add(S a, R delta, double L, float, float)
    {
        double x = a + (double)delta;
        x -= L * floor(x / L);
        return (x >= L || x < 0.0) ? 0.0 : x;
    }
};

template <class R> struct PosT<PM_FIX, R> {  // 30-bit fixed point per box edge
    typedef int S;
    __device__ static R rel(S a, S b, double, float scale, float) { return (R)fix_minimg(a - b) * (R)scale; }
    __device__ static S add(S a, R delta, double, float, float inv)
    {
        const int dq = __float2int_rn((float)delta * inv);
        return (int)(((unsigned)a + (unsigned)dq) & ((1u << kFixBits) - 1u));
    }
};

template <class R> struct PosT<PM_FREE, R> {  // unbounded (external potentials)
    typedef R S;
    __device__ static R rel(S a, S b, double, float, float) { return a - b; }
    __device__ static S add(S a, R delta, double, float, float) { return a + delta; }
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
    __device__ float value() const { return __fadd_rn(hi, lo); }
};

// plain accumulator with the same interface (FP64 form)
struct DD {
    double hi;
    __device__ void add(double x) { hi += x; }
    __device__ void warp_reduce() { hi = warp_sum(hi); }
    __device__ double value() const { return hi; }
};

// CTA-wide sum of kNQ doubles held by lane 0 of each warp into out[0..kNQ)
__device__ void cta_store_partials(const double *acc, double (*red)[kNQ], double *out)
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

// ---------------------------------------------------------------------------
// Integrator: B(dt/2) in bead space, then A(dt/2) O A(dt/2) in normal-mode
// space, one thread per (system, Cartesian component, atom).

template <int P, int PM, class R>
__global__ void __launch_bounds__(128) k_integrate(Dev d, int j)
{
    constexpr int UN = (P <= 8) ? P : 1;  // full unroll only for small rings
    __shared__ R Cs[P * P];
    __shared__ double red[4][kNQ];
    const int cta = blockIdx.x;
    const int s = d.icta_sys[cta];
    const DSys S = d.sys[s];
    if (S.P != P) return;  // another instantiation handles this system
    for (int t = threadIdx.x; t < P * P; t += blockDim.x) Cs[t] = reinterpret_cast<const R *>(d.nmC)[S.nm0 + t];
    __syncthreads();
    const int N = S.N;
    const int local = (cta - S.icta0) * blockDim.x + threadIdx.x;
    double acc[kNQ];
    for (int q = 0; q < kNQ; ++q) acc[q] = 0.0;
    double spring = 0.0;
    if (local < 3 * N) {
        typedef typename PosT<PM, R>::S PS;
        PS *X = reinterpret_cast<PS *>(d.x);
        R *V = reinterpret_cast<R *>(d.v);
        const R *F = reinterpret_cast<const R *>(d.f);
        const size_t G = (size_t)d.G;
        const int c = local / N, i = local - c * N;
        const int t = d.typ[S.g0 + i];
        const R hdtm = reinterpret_cast<const R *>(d.hdt_m)[t];
        const R sig = reinterpret_cast<const R *>(d.osig)[s * kMaxTypes + t];
        const double L = S.box[c];
        const float fsc = S.fix_scale[c], finv = S.fix_inv[c];
        const size_t base = c * G + S.g0 + i;
        const PS x0 = X[base];
        R a[P], q[P];
        // relative bead positions -> modes
#pragma unroll(UN)
        for (int b = 0; b < P; ++b)
            a[b] = (b == 0) ? R(0) : PosT<PM, R>::rel(X[base + (size_t)b * N], x0, L, fsc, finv);
#pragma unroll(UN)
        for (int k = 0; k < P; ++k) {
            R u = 0;
#pragma unroll(UN)
            for (int b = 0; b < P; ++b) u += Cs[b * P + k] * a[b];
            q[k] = u;
        }
        // B: half kick with the current forces, bead velocities -> modes
#pragma unroll(UN)
        for (int b = 0; b < P; ++b) a[b] = V[base + (size_t)b * N] + hdtm * F[base + (size_t)b * N];
        R p[P];
#pragma unroll(UN)
        for (int k = 0; k < P; ++k) {
            R u = 0;
#pragma unroll(UN)
            for (int b = 0; b < P; ++b) u += Cs[b * P + k] * a[b];
            p[k] = u;
        }
        const R *rot = reinterpret_cast<const R *>(d.rot) + 3 * S.rot0;
        const R *eta = reinterpret_cast<const R *>(d.eta) + (size_t)j * d.Dtot + S.dof0;
        const R c1 = sizeof(R) == 4 ? (R)S.c1_f : (R)S.c1;
#pragma unroll(UN)
        for (int k = 0; k < P; ++k) {
            const R cs = rot[3 * k], sw = rot[3 * k + 1], ws = rot[3 * k + 2];
            R qk = q[k], pk = p[k];
            R qn = qk * cs + pk * sw;        // A(dt/2): exact free ring-polymer rotation
            R pn = qk * ws + pk * cs;
            pn = c1 * pn + sig * eta[(size_t)(k * 3 + c) * N + i];  // O(dt)
            q[k] = qn * cs + pn * sw;        // A(dt/2)
            p[k] = qn * ws + pn * cs;
        }
        // modes -> beads
#pragma unroll(UN)
        for (int b = 0; b < P; ++b) {
            R u = 0, w = 0;
#pragma unroll(UN)
            for (int k = 0; k < P; ++k) {
                u += Cs[b * P + k] * q[k];
                w += Cs[b * P + k] * p[k];
            }
            a[b] = u;
            V[base + (size_t)b * N] = w;
        }
#pragma unroll(UN)
        for (int b = 0; b < P; ++b) X[base + (size_t)b * N] = PosT<PM, R>::add(x0, a[b], L, fsc, finv);
        if (P > 1) {
            R sp = 0;
#pragma unroll(UN)
            for (int b = 0; b < P; ++b) {
                R dd = a[b] - a[(b + 1) % P];
                sp += dd * dd;
            }
            spring = 0.5 * d.mass_mvv[t] * S.wP * S.wP * (double)sp;
        }
    }
    spring = warp_sum(spring);
    acc[Q_SPRING] = spring;
    cta_store_partials(acc, red, d.ipart + (size_t)cta * kNQ);
}

// ---------------------------------------------------------------------------
// Cell list: bin (atomic slots), then one warp per cell sorts its slots by
// bead-atom index so that every later sum has a fixed order.

template <int PM>
__global__ void k_bin(Dev d)
{
    const DRep R = d.rep[blockIdx.y];
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= R.N) return;
    const size_t G = (size_t)d.G;
    const long long g = R.g0 + i;
    int cc[3];
    for (int c = 0; c < 3; ++c) {
        int v;
        if (PM == PM_FIX) {
            unsigned xq = (unsigned)reinterpret_cast<const int *>(d.x)[c * G + g];
            v = (int)(((unsigned long long)xq * (unsigned)R.nc[c]) >> kFixBits);
        } else {
            double x = reinterpret_cast<const double *>(d.x)[c * G + g];
            v = (int)floor(x / R.box[c] * R.nc[c]);
        }
        cc[c] = min(max(v, 0), R.nc[c] - 1);
    }
    const int cell = R.cell0 + cc[0] + R.nc[0] * (cc[1] + R.nc[1] * cc[2]);
    const int slot = atomicAdd(&d.cnt[cell], 1);
    if (slot < d.cap)
        d.cidx[(size_t)cell * d.cap + slot] = (int)g;
    else
        atomicOr(d.err, (unsigned)ERR_OVERFLOW);
}

template <int PM>
__global__ void k_cellsort(Dev d)
{
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int cell = blockIdx.x * (blockDim.x >> 5) + warp;
    if (cell >= d.ncells) return;
    constexpr int E = 16;  // cap <= 512
    const int n = min(d.cnt[cell], d.cap);
    const int ne = (n + 31) >> 5;
    int key[E], rank[E];
#pragma unroll
    for (int e = 0; e < E; ++e) {
        int idx = lane + 32 * e;
        key[e] = (idx < n) ? d.cidx[(size_t)cell * d.cap + idx] : INT_MAX;
        rank[e] = 0;
    }
    for (int e2 = 0; e2 < ne; ++e2) {
        int kv = 0;
#pragma unroll
        for (int e = 0; e < E; ++e)
            if (e == e2) kv = key[e];
        for (int l = 0; l < 32; ++l) {
            const int other = __shfl_sync(0xffffffffu, kv, l);
#pragma unroll
            for (int e = 0; e < E; ++e)
                if (e < ne) rank[e] += (other < key[e]) ? 1 : 0;
        }
    }
    __syncwarp();
    const size_t G = (size_t)d.G;
#pragma unroll
    for (int e = 0; e < E; ++e) {
        int idx = lane + 32 * e;
        if (idx < n) {
            int g = key[e];
            size_t o = (size_t)cell * d.cap + rank[e];
            d.cidx[o] = g;
            if (PM == PM_FIX) {
                const int *X = reinterpret_cast<const int *>(d.x);
                reinterpret_cast<int4 *>(d.cpos)[o] = make_int4(X[g], X[G + g], X[2 * G + g], d.typ[g]);
            } else {
                const double *X = reinterpret_cast<const double *>(d.x);
                reinterpret_cast<D4 *>(d.cpos)[o] = D4{X[g], X[G + g], X[2 * G + g], (double)d.typ[g]};
            }
        }
    }
    __syncwarp();
    if (lane == 0) {
        d.ccount[cell] = n;
        d.cnt[cell] = 0;
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

// -dV/dr / r and V of one pair at squared distance r2 < rc^2, FP32 form:
// branch-free, 1/r from rsqrt + one Newton step, exponentials through exp2,
// erfc(x) = exp(-x^2) P(u) with the fitted polynomial of the table.
__device__ __forceinline__ void pair_eval(const PairTabT<float> &T, int tij, float r2, float &f_over_r, float &e,
                                          bool energy = true)
{
    float rinv = rsqrtf(r2);
    rinv = rinv * fmaf(-0.5f * r2, rinv * rinv, 1.5f);
    const float r = r2 * rinv;
    const float r2i = rinv * rinv;
    const float r6i = r2i * r2i * r2i;
    const float ex = exp2f(-r * T.inv_rho_l2e[tij]);        // exp(-r/rho); A = 0 rows give 0 below
    float f = T.A_over_rho[tij] * ex - T.C6[tij] * r6i * rinv;
    const float gg = exp2f(-T.alpha2_l2e * r2);              // exp(-alpha^2 r^2)
    const float u = fmaf(T.alpha * r, T.erfc_us, -1.0f);
    float P = T.erfc_c[11];
#pragma unroll
    for (int k = 10; k >= 0; --k) P = fmaf(P, u, T.erfc_c[k]);
    const float er = gg * P;                                  // erfc(alpha r)
    const float qq = T.qq[tij];
    f += qq * (er * r2i + T.two_a_sqrtpi * gg * rinv - T.fshift);
    f_over_r = f * rinv;
    if (energy)
        e = T.A[tij] * ex - T.C[tij] * r6i - T.eshift[tij] +
            qq * (er * rinv - T.erfc_rc_over_rc + T.fshift * (r - T.rc));
    else
        e = 0.0f;
}

// FP64 form: library exp / erfc / sqrt (the reference-accuracy path)
template <class R>
__device__ __forceinline__ void pair_eval(const PairTabT<R> &T, int tij, R r2, R &f_over_r, R &e, bool energy = true)
{
    const R r = my_sqrt(r2);
    const R rinv = R(1) / r;
    R f = 0, en = 0;
    const R A = T.A[tij], Cc = T.C[tij];
    if (A != R(0)) {
        const R ex = my_exp(-r * T.inv_rho[tij]);
        f += T.A_over_rho[tij] * ex;
        en += A * ex;
    }
    if (Cc != R(0)) {
        const R r2i = rinv * rinv;
        const R r6i = r2i * r2i * r2i;
        f -= T.C6[tij] * r6i * rinv;
        en -= Cc * r6i;
    }
    en -= T.eshift[tij];
    const R qq = T.qq[tij];
    if (qq != R(0)) {
        const R er = my_erfc(T.alpha * r);
        const R gg = my_exp(-T.alpha2 * r2);
        f += qq * (er * rinv * rinv + T.two_a_sqrtpi * gg * rinv - T.fshift);
        en += qq * (er * rinv - T.erfc_rc_over_rc + T.fshift * (r - T.rc));
    }
    f_over_r = f * rinv;
    e = en;
}

template <int PM, class R>
__global__ void __launch_bounds__(32 * kWarpsPerForceCta) k_force_pair(Dev d, PairTabT<R> T, int kick)
{
    typedef typename std::conditional<sizeof(R) == 4, float4, D4>::type R4;
    typedef typename std::conditional<sizeof(R) == 4, FF, DD>::type ACC;
    __shared__ R4 qbuf[kWarpsPerForceCta][64];
    __shared__ double red[kWarpsPerForceCta][kNQ];
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int cell = blockIdx.x / d.cpc, chunk = blockIdx.x - cell * d.cpc;
    const DRep RP = d.rep[d.cell_rep[cell]];
    const int cnt = d.ccount[cell];
    const int slot = chunk * kWarpsPerForceCta + warp;
    double acc[kNQ];
#pragma unroll
    for (int q = 0; q < kNQ; ++q) acc[q] = 0.0;
    if (slot < cnt) {
        const size_t hoff = (size_t)cell * d.cap + slot;
        const int gi = d.cidx[hoff];
        R hx = 0, hy = 0, hz = 0;
        int ti;
        int ihx = 0, ihy = 0, ihz = 0;
        if (PM == PM_FIX) {
            int4 hp = reinterpret_cast<const int4 *>(d.cpos)[hoff];
            ihx = hp.x; ihy = hp.y; ihz = hp.z; ti = hp.w;
        } else {
            D4 hp = reinterpret_cast<const D4 *>(d.cpos)[hoff];
            hx = (R)hp.x; hy = (R)hp.y; hz = (R)hp.z; ti = (int)hp.w;
        }
        const int lc = cell - RP.cell0;
        const int cx = lc % RP.nc[0], cy = (lc / RP.nc[0]) % RP.nc[1], cz = lc / (RP.nc[0] * RP.nc[1]);
        const R sx = (R)RP.fix_scale[0], sy = (R)RP.fix_scale[1], sz = (R)RP.fix_scale[2];
        const R rc2 = T.rc2;
        ACC fx{}, fy{}, fz{};
        R en = 0, w0 = 0, w1 = 0, w2 = 0, w3 = 0, w4 = 0, w5 = 0;
        int qn = 0;
        R4 *qb = qbuf[warp];
        const unsigned lt = (1u << lane) - 1u;
        auto consume = [&](int m) {
            if (lane < m) {
                R4 e4 = qb[lane];
                int tj;
                if (sizeof(R) == 4) tj = __float_as_int((float)e4.w); else tj = (int)e4.w;
                R r2 = e4.x * e4.x + e4.y * e4.y + e4.z * e4.z;
                R fo, ee;
                pair_eval<R>(T, ti * kMaxTypes + tj, r2, fo, ee);
                // stored displacement is r_j - r_i: the force on i is -fo (r_j - r_i)
                fx.add(-fo * e4.x); fy.add(-fo * e4.y); fz.add(-fo * e4.z);
                en += ee;
                w0 += fo * e4.x * e4.x; w1 += fo * e4.y * e4.y; w2 += fo * e4.z * e4.z;
                w3 += fo * e4.x * e4.y; w4 += fo * e4.x * e4.z; w5 += fo * e4.y * e4.z;
            }
        };
        for (int oz = -1; oz <= 1; ++oz)
            for (int oy = -1; oy <= 1; ++oy)
                for (int ox = -1; ox <= 1; ++ox) {
                    int ux = cx + ox, uy = cy + oy, uz = cz + oz;
                    const int mx = (int)floor_div(ux, RP.nc[0]), my = (int)floor_div(uy, RP.nc[1]),
                              mz = (int)floor_div(uz, RP.nc[2]);
                    ux -= mx * RP.nc[0]; uy -= my * RP.nc[1]; uz -= mz * RP.nc[2];
                    const int nc = RP.cell0 + ux + RP.nc[0] * (uy + RP.nc[1] * uz);
                    const int ncnt = d.ccount[nc];
                    const bool selfc = (ox == 0 && oy == 0 && oz == 0);
                    const size_t nb = (size_t)nc * d.cap;
                    for (int e0 = 0; e0 < ncnt; e0 += 32) {
                        const int e = e0 + lane;
                        R dx = 0, dy = 0, dz = 0;
                        int tj = 0;
                        bool take = false;
                        if (e < ncnt && !(selfc && e == slot)) {
                            if (PM == PM_FIX) {
                                int4 pj = reinterpret_cast<const int4 *>(d.cpos)[nb + e];
                                // displacement r_j + image - r_i, exact in int32
                                const int ix = (int)((unsigned)pj.x - (unsigned)ihx + (unsigned)mx * (1u << kFixBits));
                                const int iy = (int)((unsigned)pj.y - (unsigned)ihy + (unsigned)my * (1u << kFixBits));
                                const int iz = (int)((unsigned)pj.z - (unsigned)ihz + (unsigned)mz * (1u << kFixBits));
                                dx = (R)ix * sx; dy = (R)iy * sy; dz = (R)iz * sz;
                                tj = pj.w;
                            } else {
                                D4 pj = reinterpret_cast<const D4 *>(d.cpos)[nb + e];
                                dx = (R)(pj.x + mx * RP.box[0]) - hx;
                                dy = (R)(pj.y + my * RP.box[1]) - hy;
                                dz = (R)(pj.z + mz * RP.box[2]) - hz;
                                tj = (int)pj.w;
                            }
                            take = (dx * dx + dy * dy + dz * dz) < rc2;
                        }
                        const unsigned m = __ballot_sync(0xffffffffu, take);
                        if (take) {
                            R4 v;
                            v.x = dx; v.y = dy; v.z = dz;
                            if (sizeof(R) == 4) v.w = (R)__int_as_float(tj); else v.w = (R)tj;
                            qb[qn + __popc(m & lt)] = v;
                        }
                        qn += __popc(m);
                        __syncwarp();
                        if (qn >= 32) {
                            consume(32);
                            __syncwarp();
                            R4 carry;
                            if (lane < qn - 32) carry = qb[32 + lane];
                            __syncwarp();
                            if (lane < qn - 32) qb[lane] = carry;
                            qn -= 32;
                            __syncwarp();
                        }
                    }
                }
        consume(qn);
        fx.warp_reduce(); fy.warp_reduce(); fz.warp_reduce();
        en = warp_sum(en);
        w0 = warp_sum(w0); w1 = warp_sum(w1); w2 = warp_sum(w2);
        w3 = warp_sum(w3); w4 = warp_sum(w4); w5 = warp_sum(w5);
        if (lane == 0) {
            const DSys &S = d.sys[RP.sys];
            const size_t G = (size_t)d.G;
            R *Fo = reinterpret_cast<R *>(d.f);
            R *V = reinterpret_cast<R *>(d.v);
            const R invP = sizeof(R) == 4 ? (R)S.invP_f : (R)S.invP;
            const R f3[3] = {(R)fx.value() * invP, (R)fy.value() * invP, (R)fz.value() * invP};
            const R hdtm = T.hdt_m[ti];
            double ke = 0.0;
            for (int c = 0; c < 3; ++c) {
                Fo[c * G + gi] = f3[c];
                R v = V[c * G + gi];
                if (kick) {
                    v += hdtm * f3[c];
                    V[c * G + gi] = v;
                }
                ke += 0.5 * T.mass_mvv[ti] * (double)v * (double)v;
                acc[Q_MOM + c] = T.mass[ti] * (double)v;
            }
            acc[Q_K] = ke;
            acc[Q_V] = 0.5 * (double)en;
            acc[Q_VIR + 0] = 0.5 * (double)w0; acc[Q_VIR + 1] = 0.5 * (double)w1; acc[Q_VIR + 2] = 0.5 * (double)w2;
            acc[Q_VIR + 3] = 0.5 * (double)w3; acc[Q_VIR + 4] = 0.5 * (double)w4; acc[Q_VIR + 5] = 0.5 * (double)w5;
        }
    }
    cta_store_partials(acc, red, d.part + (size_t)blockIdx.x * kNQ);
}

// Per-system reduction of the CTA partials into the observable record
// (fixed summation order, FP64).  Executed by one CTA.
__device__ void reduce_system(const Dev &d, int s, long long step, int record, double (*sh)[kNQ + 1])
{
    const DSys S = d.sys[s];
    const int nt = min((int)blockDim.x, 128);  // threads taking part (a power of two)
    if ((int)threadIdx.x < nt) {
        double acc[kNQ + 1];
        for (int q = 0; q <= kNQ; ++q) acc[q] = 0.0;
        for (int c = S.fcta0 + (int)threadIdx.x; c < S.fcta1; c += nt)
            for (int q = 0; q < kNQ; ++q) acc[q] += d.part[(size_t)c * kNQ + q];
        for (int c = S.icta0 + (int)threadIdx.x; c < S.icta1; c += nt) acc[kNQ] += d.ipart[(size_t)c * kNQ + Q_SPRING];
        for (int q = 0; q <= kNQ; ++q) sh[threadIdx.x][q] = acc[q];
    }
    __syncthreads();
    for (int w = nt / 2; w > 0; w >>= 1) {
        if ((int)threadIdx.x < w)
            for (int q = 0; q <= kNQ; ++q) sh[threadIdx.x][q] += sh[threadIdx.x + w][q];
        __syncthreads();
    }
    if (threadIdx.x == 0) {
        const double invP = S.invP;
        double rec[QTB_NREC];
        for (int q = 0; q < QTB_NREC; ++q) rec[q] = 0.0;
        const double K = sh[0][Q_K], V = sh[0][Q_V] * invP, sp = sh[0][kNQ];
        rec[0] = (double)step;
        rec[1] = K;
        rec[2] = V;
        rec[3] = sp;
        rec[4] = K - sp + V;
        const int map[9] = {0, 3, 4, 3, 1, 5, 4, 5, 2};  // xx xy xz / yx yy yz / zx zy zz
        for (int a = 0; a < 9; ++a) rec[5 + a] = sh[0][Q_VIR + map[a]] * invP;
        for (int c = 0; c < 3; ++c) rec[14 + c] = sh[0][Q_MOM + c];
        rec[17] = sh[0][Q_X2] * invP;
        if (!isfinite(K) || !isfinite(V)) atomicOr(d.err, (unsigned)ERR_NONFINITE);
        for (int q = 0; q < QTB_NREC; ++q) d.latest[(size_t)s * QTB_NREC + q] = rec[q];
        if (record >= 0 && step % d.obs_stride == 0) {
            long long r = step / d.obs_stride - 1;
            int slot = (int)(r % d.max_records);
            for (int q = 0; q < QTB_NREC; ++q) d.series[((size_t)slot * d.nsys + s) * QTB_NREC + q] = rec[q];
        }
    }
}

// Pair force with the neighbourhood staged in shared memory.
// Cells are >= r_c / 2, the stencil is the 5^3 surrounding cells (with
// explicit periodic images).  One CTA per home cell: its warps stage every
// stencil cell (sorted slots, image shift already added: fixed point + m 2^30
// stays inside int32 because positions are < 2^30), then each warp takes one
// home atom at a time and scans the flat staged array, compacting the pairs
// within r_c into a shared-memory queue that all 32 lanes evaluate together.
// Energies, virials and kinetic energies are formed only on recorded steps;
// the last CTA of a system to finish then reduces the system's partials.
constexpr int kStencilHalf = 2;
constexpr int kStencil = (2 * kStencilHalf + 1) * (2 * kStencilHalf + 1) * (2 * kStencilHalf + 1);

template <int PM, class R>
__global__ void __launch_bounds__(32 * kWarpsPerForceCta, sizeof(R) == 4 ? 3 : 1)
    k_force_cells(Dev d, PairTabT<R> T, int kick, int j)
{
    typedef typename std::conditional<sizeof(R) == 4, float4, D4>::type R4;
    typedef typename std::conditional<PM == PM_FIX, int4, D4>::type E4;
    typedef typename std::conditional<sizeof(R) == 4, FF, DD>::type ACC;
    constexpr int SH = kStencilHalf, SW = 2 * kStencilHalf + 1;
    extern __shared__ __align__(32) unsigned char fsm[];
    __shared__ R4 qbuf[kWarpsPerForceCta][128];
    __shared__ double red[kWarpsPerForceCta][kNQ];
    __shared__ int soff[kStencil + 1], scell[kStencil], simg[kStencil][3];
    __shared__ int s_last;
    E4 *stage = reinterpret_cast<E4 *>(fsm);
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int cell = blockIdx.x;
    const int cnt = d.ccount[cell];
    const long long step = d.clock[0] * kBlockSteps + j + 1;
    const bool rec = (kick == 0) || (step % d.obs_stride == 0);
    const DRep RP = d.rep[d.cell_rep[cell]];
    double acc[kNQ];
#pragma unroll
    for (int q = 0; q < kNQ; ++q) acc[q] = 0.0;
    if (cnt > 0) {
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
        // capacity of the staging buffer (sentinel padding to a multiple of 64 included)
        int total = soff[kStencil];
        if (((total + 63) & ~63) > d.stage_cap) {
            if (threadIdx.x == 0) atomicOr(d.err, (unsigned)ERR_OVERFLOW);
            total = (d.stage_cap & ~63);
        }
        const int padded = (total + 63) & ~63;
        // flat staging: every thread first issues all of its (independent) loads,
        // then shifts by the image and stores, so the CTA pays one memory latency
        {
            constexpr int U = 8;  // entries per thread per round (2048 per round for 256 threads)
            for (int base = 0; base < total; base += U * (int)blockDim.x) {
                E4 buf[U];
                int tcell[U], dst[U];
#pragma unroll
                for (int u = 0; u < U; ++u) {
                    const int e = base + u * (int)blockDim.x + (int)threadIdx.x;
                    dst[u] = -1;
                    tcell[u] = 0;
                    if (e < total) {
                        int lo = 0, hi = kStencil - 1;  // stencil cell t with soff[t] <= e < soff[t+1]
                        while (lo < hi) {
                            const int mid = (lo + hi + 1) >> 1;
                            if (soff[mid] <= e) lo = mid; else hi = mid - 1;
                        }
                        tcell[u] = lo;
                        dst[u] = e;
                        buf[u] = reinterpret_cast<const E4 *>(d.cpos)[(size_t)scell[lo] * d.cap + (e - soff[lo])];
                    }
                }
#pragma unroll
                for (int u = 0; u < U; ++u) {
                    if (dst[u] < 0) continue;
                    E4 p = buf[u];
                    const int t = tcell[u];
                    if (PM == PM_FIX) {
                        p.x = (int)((unsigned)p.x + (unsigned)simg[t][0] * (1u << kFixBits));
                        p.y = (int)((unsigned)p.y + (unsigned)simg[t][1] * (1u << kFixBits));
                        p.z = (int)((unsigned)p.z + (unsigned)simg[t][2] * (1u << kFixBits));
                    } else {
                        p.x += simg[t][0] * RP.box[0];
                        p.y += simg[t][1] * RP.box[1];
                        p.z += simg[t][2] * RP.box[2];
                    }
                    stage[dst[u]] = p;
                }
            }
        }
        // sentinel entries far outside r_cut pad the scan to a multiple of 64
        for (int e = total + threadIdx.x; e < padded; e += blockDim.x) {
            if (PM == PM_FIX) reinterpret_cast<int4 *>(stage)[e] = make_int4(-(1 << kFixBits), -(1 << kFixBits), -(1 << kFixBits), 0);
            else reinterpret_cast<D4 *>(stage)[e] = D4{-1e30, -1e30, -1e30, 0.0};
        }
        __syncthreads();
        const int self0 = soff[kStencil / 2];  // stencil offset (0,0,0)
        const R sx = (R)RP.fix_scale[0], sy = (R)RP.fix_scale[1], sz = (R)RP.fix_scale[2];
        const R rc2 = T.rc2;
        const DSys &S = d.sys[RP.sys];
        const R invP = sizeof(R) == 4 ? (R)S.invP_f : (R)S.invP;
        const unsigned lt = (1u << lane) - 1u;
        R4 *qb = qbuf[warp];  // ring of 128 queued pairs
        for (int slot = warp; slot < cnt; slot += kWarpsPerForceCta) {
            const E4 hp = stage[self0 + slot];
            int ti;
            if (PM == PM_FIX) ti = hp.w; else ti = (int)hp.w;
            ACC fx{}, fy{}, fz{};
            R en = 0, w0 = 0, w1 = 0, w2 = 0, w3 = 0, w4 = 0, w5 = 0;
            int qh = 0, qn = 0;  // ring head, queued count
            auto consume = [&](int m) {
                if (lane < m) {
                    R4 e4 = qb[(qh + lane) & 127];
                    int tj;
                    if (sizeof(R) == 4) tj = __float_as_int((float)e4.w); else tj = (int)e4.w;
                    R r2 = e4.x * e4.x + e4.y * e4.y + e4.z * e4.z;
                    R fo, ee;
                    pair_eval<R>(T, ti * kMaxTypes + tj, r2, fo, ee, rec);
                    // stored displacement is r_j - r_i: the force on i is -fo (r_j - r_i)
                    fx.add(-fo * e4.x); fy.add(-fo * e4.y); fz.add(-fo * e4.z);
                    if (rec) {
                        en += ee;
                        w0 += fo * e4.x * e4.x; w1 += fo * e4.y * e4.y; w2 += fo * e4.z * e4.z;
                        w3 += fo * e4.x * e4.y; w4 += fo * e4.x * e4.z; w5 += fo * e4.y * e4.z;
                    }
                }
            };
            auto disp = [&](const E4 &pj, R &dx, R &dy, R &dz) {
                if (PM == PM_FIX) {
                    dx = (R)(int)((unsigned)pj.x - (unsigned)hp.x) * sx;
                    dy = (R)(int)((unsigned)pj.y - (unsigned)hp.y) * sy;
                    dz = (R)(int)((unsigned)pj.z - (unsigned)hp.z) * sz;
                } else {
                    dx = (R)(pj.x - hp.x);
                    dy = (R)(pj.y - hp.y);
                    dz = (R)(pj.z - hp.z);
                }
            };
            auto push = [&](bool take, R dx, R dy, R dz, int tj) {
                const unsigned m = __ballot_sync(0xffffffffu, take);
                if (take) {
                    R4 v;
                    v.x = dx; v.y = dy; v.z = dz;
                    if (sizeof(R) == 4) v.w = (R)__int_as_float(tj); else v.w = (R)tj;
                    qb[(qh + qn + __popc(m & lt)) & 127] = v;
                }
                qn += __popc(m);
            };
            // two independent candidates per lane per iteration; the home atom
            // itself (r2 == 0) and the sentinels (r2 >= rc2) fail the test
            for (int e0 = 0; e0 < padded; e0 += 64) {
                const E4 pa = stage[e0 + lane], pb = stage[e0 + 32 + lane];
                R ax, ay, az, bx, by, bz;
                disp(pa, ax, ay, az);
                disp(pb, bx, by, bz);
                const R ra = ax * ax + ay * ay + az * az, rb = bx * bx + by * by + bz * bz;
                int ta, tb;
                if (PM == PM_FIX) { ta = pa.w; tb = pb.w; } else { ta = (int)pa.w; tb = (int)pb.w; }
                push(ra < rc2 && ra > R(0), ax, ay, az, ta);
                push(rb < rc2 && rb > R(0), bx, by, bz, tb);
                __syncwarp();
                while (qn >= 32) {
                    consume(32);
                    qh = (qh + 32) & 127;
                    qn -= 32;
                }
                __syncwarp();
            }
            consume(qn);
            __syncwarp();
            fx.warp_reduce(); fy.warp_reduce(); fz.warp_reduce();
            if (rec) {
                en = warp_sum(en);
                w0 = warp_sum(w0); w1 = warp_sum(w1); w2 = warp_sum(w2);
                w3 = warp_sum(w3); w4 = warp_sum(w4); w5 = warp_sum(w5);
            }
            if (lane == 0) {
                const int gi = d.cidx[(size_t)cell * d.cap + slot];
                const size_t G = (size_t)d.G;
                R *Fo = reinterpret_cast<R *>(d.f);
                R *V = reinterpret_cast<R *>(d.v);
                const R f3[3] = {(R)fx.value() * invP, (R)fy.value() * invP, (R)fz.value() * invP};
                const R hdtm = T.hdt_m[ti];
                R v3[3];
                for (int c = 0; c < 3; ++c) {
                    Fo[c * G + gi] = f3[c];
                    R v = V[c * G + gi];
                    if (kick) {
                        v += hdtm * f3[c];
                        V[c * G + gi] = v;
                    }
                    v3[c] = v;
                }
                if (rec) {
                    double ke = 0.0;
                    for (int c = 0; c < 3; ++c) {
                        ke += 0.5 * T.mass_mvv[ti] * (double)v3[c] * (double)v3[c];
                        acc[Q_MOM + c] += T.mass[ti] * (double)v3[c];
                    }
                    acc[Q_K] += ke;
                    acc[Q_V] += 0.5 * (double)en;
                    acc[Q_VIR + 0] += 0.5 * (double)w0; acc[Q_VIR + 1] += 0.5 * (double)w1;
                    acc[Q_VIR + 2] += 0.5 * (double)w2; acc[Q_VIR + 3] += 0.5 * (double)w3;
                    acc[Q_VIR + 4] += 0.5 * (double)w4; acc[Q_VIR + 5] += 0.5 * (double)w5;
                }
            }
        }
    }
    if (!rec) return;
    cta_store_partials(acc, red, d.part + (size_t)blockIdx.x * kNQ);
    // last CTA of this system reduces (partials made visible first)
    __threadfence();
    __syncthreads();
    if (threadIdx.x == 0) {
        const DSys &S = d.sys[RP.sys];
        const unsigned prev = atomicAdd(&d.done[RP.sys], 1u);
        s_last = (prev == (unsigned)(S.fcta1 - S.fcta0 - 1)) ? 1 : 0;
    }
    __syncthreads();
    if (s_last) {
        __threadfence();
        // the staging buffer is free now: reuse it for the reduction
        reduce_system(d, RP.sys, step, kick ? 1 : -1, reinterpret_cast<double (*)[kNQ + 1]>(fsm));
        if (threadIdx.x == 0) d.done[RP.sys] = 0u;
    }
}

template <int PM, class R> size_t force_cells_smem(int entries)
{
    typedef typename std::conditional<PM == PM_FIX, int4, D4>::type E4;
    const size_t stage = (size_t)entries * sizeof(E4);
    const size_t redn = (size_t)128 * (kNQ + 1) * sizeof(double);
    return stage > redn ? stage : redn;
}

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
    cta_store_partials(acc, red, d.part + ((size_t)blockIdx.y * gridDim.x + blockIdx.x) * kNQ);
}

// ---------------------------------------------------------------------------
// Per-system reduction into the observable record (fixed summation order).

__global__ void k_reduce(Dev d, int j, int record)
{
    __shared__ double sh[128][kNQ + 1];
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

template <int PM, class R>
static void integrate_all(const Dev &d, const MdLaunch &m, int j, cudaStream_t st)
{
    for (int u = 0; u < m.nP; ++u) {
        switch (m.Pvals[u]) {
#define QTB_P(PP) case PP: k_integrate<PP, PM, R><<<m.n_icta, 128, 0, st>>>(d, j); break;
            QTB_P(1) QTB_P(2) QTB_P(3) QTB_P(4) QTB_P(5) QTB_P(6) QTB_P(8) QTB_P(16) QTB_P(32)
#undef QTB_P
            default: break;
        }
    }
}

void launch_integrate(const Dev &d, const MdLaunch &m, int j, cudaStream_t st)
{
    if (!m.pair) {
        if (m.mixed) integrate_all<PM_FREE, float>(d, m, j, st);
        else integrate_all<PM_FREE, double>(d, m, j, st);
    } else {
        if (m.mixed) integrate_all<PM_FIX, float>(d, m, j, st);
        else integrate_all<PM_BOX64, double>(d, m, j, st);
    }
}

void launch_cells(const Dev &d, const MdLaunch &m, cudaStream_t st)
{
    if (!m.pair) return;
    dim3 g((unsigned)m.n_bcta, (unsigned)d.nrep);
    if (m.mixed) {
        k_bin<PM_FIX><<<g, 256, 0, st>>>(d);
        k_cellsort<PM_FIX><<<(d.ncells + 7) / 8, 256, 0, st>>>(d);
    } else {
        k_bin<PM_BOX64><<<g, 256, 0, st>>>(d);
        k_cellsort<PM_BOX64><<<(d.ncells + 7) / 8, 256, 0, st>>>(d);
    }
}

size_t force_staged_smem(int cap, int mixed)
{
    return mixed ? force_cells_smem<PM_FIX, float>(cap) : force_cells_smem<PM_BOX64, double>(cap);
}

cudaError_t force_staged_prepare(int cap, int mixed)
{
    const int sm = (int)force_staged_smem(cap, mixed);
    if (mixed) return cudaFuncSetAttribute(k_force_cells<PM_FIX, float>, cudaFuncAttributeMaxDynamicSharedMemorySize, sm);
    return cudaFuncSetAttribute(k_force_cells<PM_BOX64, double>, cudaFuncAttributeMaxDynamicSharedMemorySize, sm);
}

void launch_force_kick(const Dev &d, const MdLaunch &m, const PairTabT<float> &Tf, const PairTabT<double> &Td,
                       int kick, int j, cudaStream_t st)
{
    if (m.pair && m.staged) {
        const unsigned grid = (unsigned)d.ncells;
        const size_t sm = force_staged_smem(d.stage_cap, m.mixed);
        if (m.mixed) k_force_cells<PM_FIX, float><<<grid, 32 * kWarpsPerForceCta, sm, st>>>(d, Tf, kick, j);
        else k_force_cells<PM_BOX64, double><<<grid, 32 * kWarpsPerForceCta, sm, st>>>(d, Td, kick, j);
    } else if (m.pair) {
        const unsigned grid = (unsigned)(d.ncells * d.cpc);
        if (m.mixed) k_force_pair<PM_FIX, float><<<grid, 32 * kWarpsPerForceCta, 0, st>>>(d, Tf, kick);
        else k_force_pair<PM_BOX64, double><<<grid, 32 * kWarpsPerForceCta, 0, st>>>(d, Td, kick);
    } else {
        dim3 g((unsigned)m.n_ecta, (unsigned)d.nsys);
        if (m.mixed) k_force_ext<float><<<g, 128, 0, st>>>(d, Tf, kick);
        else k_force_ext<double><<<g, 128, 0, st>>>(d, Td, kick);
    }
}

void launch_reduce(const Dev &d, const MdLaunch &m, int j, int record, cudaStream_t st)
{
    k_reduce<<<d.nsys, 128, 0, st>>>(d, j, record);
}

void launch_tick(const Dev &d, cudaStream_t st) { k_tick<<<1, 1, 0, st>>>(d); }
void launch_setclock(const Dev &d, long long b, cudaStream_t st) { k_setclock<<<1, 1, 0, st>>>(d, b); }

}  // namespace qtb
