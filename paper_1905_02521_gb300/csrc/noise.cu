// noise.cu -- white noise, SIMT noise filters, spectra, filter taps and the
// FP64 kappa_P solve of the QTB / QTB-PIMD random force (sm_103a).
//
// Eqs. 6-7: the random force has spectral density 2 m gamma theta(w,T);
// Eq. 12: QTB-PIMD uses kappa_P (Eq. 10) instead.  The force of the O step is
// sqrt((1-c1^2)/m) eta_n, eta_n = sum_{k=-K..K} h_|k| xi_{n-k}: a zero-phase
// time-domain filter of counter-based white noise xi whose response equals
// sqrt(S(w_j)) on the grid w_j = 2 pi j/(L dt), S = theta W or kappa_P W.
#include <cuda_bf16.h>

#include <algorithm>

#include "qtb_dev.cuh"
#include "qtb_kernels.cuh"

namespace qtb {

// ---------------------------------------------------------------------------
// White noise: one Philox call per (dof, 4 steps); Box-Muller pairs
// (w0,w1) -> steps 4q, 4q+1 (cos, sin), (w2,w3) -> 4q+2, 4q+3.

__device__ __forceinline__ void bm_pair(uint32_t a, uint32_t b, double &z0, double &z1)
{
    double u1 = ((double)a + 1.0) * 2.3283064365386963e-10;  // 2^-32, (0, 1]
    double u2 = (double)b * 2.3283064365386963e-10;          // [0, 1)
    double r = sqrt(-2.0 * log(u1));
    double s, c;
    sincospi(2.0 * u2, &s, &c);
    z0 = r * c;
    z1 = r * s;
}

__device__ __forceinline__ void bm_pair(uint32_t a, uint32_t b, float &z0, float &z1)
{
    float u1 = ((float)a + 1.0f) * 2.3283064365386963e-10f;
    float u2 = (float)b * 2.3283064365386963e-10f;
    float r = sqrtf(-2.0f * logf(u1));
    float s, c;
    sincospif(2.0f * u2, &s, &c);
    z0 = r * c;
    z1 = r * s;
}

template <class T> struct RingStore;
template <> struct RingStore<double> {
    __device__ static void put(double *p, double a, double b, double c, double d)
    {
        reinterpret_cast<double2 *>(p)[0] = make_double2(a, b);
        reinterpret_cast<double2 *>(p)[1] = make_double2(c, d);
    }
};
template <> struct RingStore<float> {
    __device__ static void put(float *p, float a, float b, float c, float d)
    {
        *reinterpret_cast<float4 *>(p) = make_float4(a, b, c, d);
    }
};
template <> struct RingStore<__nv_bfloat16> {
    __device__ static void put(__nv_bfloat16 *p, float a, float b, float c, float d)
    {
        __nv_bfloat162 lo = __floats2bfloat162_rn(a, b), hi = __floats2bfloat162_rn(c, d);
        uint2 u;
        u.x = *reinterpret_cast<uint32_t *>(&lo);
        u.y = *reinterpret_cast<uint32_t *>(&hi);
        *reinterpret_cast<uint2 *>(p) = u;
    }
};

// Generate white block `blk` (blk_abs >= -2^40; blk_override == LLONG_MIN means
// clock + Kb) into its ring slot.  grid = (ceil(max dofp * 64 / 256), nsys).
template <class T, class C>
__global__ void k_white(Dev d, long long blk_override)
{
    const DSys s = d.sys[blockIdx.y];
    long long local = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    int dofl = (int)(local >> 6), qi = (int)(local & 63);
    if (dofl >= s.dofp) return;
    long long blk = (blk_override == LLONG_MIN) ? d.clock[0] + d.Kb : blk_override;
    int slot = (int)(blk - floor_div(blk, d.nslots) * d.nslots);
    T *dst = reinterpret_cast<T *>(d.ring) + ((size_t)slot * d.Dtot + s.dof0 + dofl) * kBlockSteps + 4 * qi;
    C z0 = 0, z1 = 0, z2 = 0, z3 = 0;
    if (dofl < 3 * s.N * s.P) {
        long long q = blk * (kBlockSteps / 4) + qi;
        unsigned long long uq = (unsigned long long)q;
        uint4 ctr = make_uint4((uint32_t)uq, (uint32_t)dofl, 0u, (uint32_t)(uq >> 32));
        uint32_t sysid = (uint32_t)blockIdx.y;
        uint4 w = philox4x32_10(ctr, (uint32_t)d.seed, (uint32_t)(d.seed >> 32) ^ sysid);
        bm_pair(w.x, w.y, z0, z1);
        bm_pair(w.z, w.w, z2, z3);
    }
    RingStore<T>::put(dst, z0, z1, z2, z3);
}

// ---------------------------------------------------------------------------
// SIMT filter: one CTA (256 threads = 256 output steps) per dof.
// grid = (max dofp, nsys); dynamic smem = (256 + 2 Kmax + Kmax + 1) * sizeof(T)
template <class T>
__global__ void k_filter_simt(Dev d)
{
    extern __shared__ unsigned char smraw[];
    T *win = reinterpret_cast<T *>(smraw);
    const DSys s = d.sys[blockIdx.y];
    int dofl = blockIdx.x;
    if (dofl >= s.dofp) return;
    const int K = s.K, span = kBlockSteps + 2 * K;
    T *h = win + span;
    long long blk = d.clock[0];
    T *eta = reinterpret_cast<T *>(d.eta);
    const int j = threadIdx.x;
    if (dofl >= 3 * s.N * s.P) {
        eta[(size_t)j * d.Dtot + s.dof0 + dofl] = T(0);
        return;
    }
    const T *ring = reinterpret_cast<const T *>(d.ring);
    const T *taps = reinterpret_cast<const T *>(d.tapsR) + s.taps0;
    for (int t = threadIdx.x; t < span; t += blockDim.x) {
        long long n = blk * kBlockSteps - K + t;
        long long rb = floor_div(n, kBlockSteps);
        int slot = (int)(rb - floor_div(rb, d.nslots) * d.nslots);
        win[t] = ring[((size_t)slot * d.Dtot + s.dof0 + dofl) * kBlockSteps + (int)(n - rb * kBlockSteps)];
    }
    for (int t = threadIdx.x; t <= K; t += blockDim.x) h[t] = taps[t];
    __syncthreads();
    // xi(n - k) with n = blk*256 + j sits at window index j + K - k
    T acc = h[0] * win[j + K];
    for (int k = 1; k <= K; ++k) acc += h[k] * (win[j + K - k] + win[j + K + k]);
    eta[(size_t)j * d.Dtot + s.dof0 + dofl] = acc;
}

// ---------------------------------------------------------------------------
// Spectra and taps (FP64).

__device__ double theta_dev(double w, double T)
{
    w = fabs(w);
    double kT = kBoltz * T;
    double x = kHbar * w / kT;
    if (x < 1e-6) return kT * (1.0 + x * x / 12.0);
    return kHbar * w * (0.5 + 1.0 / expm1(x));
}

__device__ double fth_dev(double x)
{
    x = fabs(x);
    if (x < 1e-6) return 1.0 + x * x / 12.0;
    return x * (0.5 + 1.0 / expm1(x));
}

__device__ double kappa_tail_dev(int P, double y)
{
    if (P == 1) return fth_dev(y);
    return fth_dev(sqrt((double)P) * y) / P + sqrt((double)P) / (2.0 * y);
}

// F_P at y from the collocation grid y_i = y0 sinh(i dts)
__device__ double kappa_eval_dev(const DSpec &sp, double y)
{
    if (sp.P == 1) return fth_dev(y);
    if (y > sp.ymax) return kappa_tail_dev(sp.P, y);
    double dts = asinh(sp.ymax / sp.y0) / (sp.n - 1);
    int i = (int)(asinh(y / sp.y0) / dts);
    if (i > sp.n - 2) i = sp.n - 2;
    double ya = sp.y0 * sinh(i * dts), yb = sp.y0 * sinh((i + 1) * dts);
    double lam = (y - ya) / (yb - ya);
    return sp.F[i] * (1.0 - lam) + sp.F[i + 1] * lam;
}

// S_j, j = 0..K, per system.  grid = (ceil((Kmax+1)/256), nsys)
// spectral density at w (rad/fs) of a system in a non-learned mode: k_B T
// (white), theta (QTB, Eq. 7) or kappa_P (QTB-PIMD, Eq. 12), times the cutoff
__device__ double spectrum_value(const DSpec &sp, double w)
{
    double base;
    if (sp.mode == QTB_NOISE_WHITE) {
        base = kBoltz * sp.T;
    } else if (sp.mode == QTB_NOISE_QTB) {
        base = theta_dev(w, sp.T);
    } else {
        double kT = kBoltz * sp.T;
        base = kT * kappa_eval_dev(sp, kHbar * w / kT);
    }
    double W = 1.0;
    if (sp.mode != QTB_NOISE_WHITE && sp.omega_max > 0.0)
        W = 1.0 / (1.0 + exp((w - sp.omega_max) / (sp.omega_max / 50.0)));
    return base * W;
}

__global__ void k_spectrum(const DSpec *spec, double *S)
{
    const DSpec sp = spec[blockIdx.y];
    int j = blockIdx.x * blockDim.x + threadIdx.x;
    if (j > sp.K) return;
    if (sp.mode == QTB_NOISE_QTB_PIMD_MLP) return;  // filled by the learned model's spectrum kernel (mlp.cu)
    int L = 2 * sp.K + 1;
    S[sp.taps0 + j] = spectrum_value(sp, 2.0 * kPi * j / (L * sp.dt));
}

__global__ void k_taps(const DSpec *spec, const double *S, double *h64, float *h32)
{
    const DSpec sp = spec[blockIdx.y];
    int k = blockIdx.x * blockDim.x + threadIdx.x;
    if (k > sp.K) return;
    const int K = sp.K;
    const long long L = 2 * K + 1;
    const double *Sj = S + sp.taps0;
    double acc = 0.0;
    for (int j = 1; j <= K; ++j) {
        long long m = ((long long)j * k) % L;
        acc += sqrt(Sj[j]) * cospi(2.0 * (double)m / (double)L);
    }
    double h = (sqrt(Sj[0]) + 2.0 * acc) / (double)L;
    h64[sp.taps0 + k] = h;
    h32[sp.taps0 + k] = (float)h;
}

// ---------------------------------------------------------------------------
// kappa_P solve (Eq. 10), FP64: dense collocation rows, normal equations,
// blocked Cholesky (many CTAs), triangular solves (one CTA), one refinement step.

// rows m < 2n-1; A is (2n-1) x n row-major, zeroed by the caller
__global__ void k_kappa_rows(int P, int n, double ymax, double y0, double *A, double *b)
{
    int m = blockIdx.x * blockDim.x + threadIdx.x;
    int rows = 2 * n - 1;
    if (m >= rows) return;
    double dts = asinh(ymax / y0) / (n - 1);
    double y = y0 * sinh(0.5 * m * dts);
    double rhs = fth_dev(sqrt((double)P) * y);
    double *Ar = A + (size_t)m * n;
    for (int k = 0; k < P; ++k) {
        double sk = sinpi((double)k / P);
        double ck = 4.0 * P * sk * sk;
        double yk = sqrt(y * y + ck);
        double w = (k == 0) ? 1.0 : ((y * y + ck) > 0.0 ? y * y / (y * y + ck) : 0.0);
        if (w == 0.0) continue;
        if (yk <= ymax) {
            int i = (int)(asinh(yk / y0) / dts);
            if (i > n - 2) i = n - 2;
            double ya = y0 * sinh(i * dts), yb = y0 * sinh((i + 1) * dts);
            double lam = (yk - ya) / (yb - ya);
            Ar[i] += w * (1.0 - lam);
            Ar[i + 1] += w * lam;
        } else {
            rhs -= w * kappa_tail_dev(P, yk);
        }
    }
    double sc = 1.0 / fth_dev(sqrt((double)P) * y);
    for (int i = 0; i < n; ++i) Ar[i] *= sc;
    b[m] = rhs * sc;
}

// M = A^T A (n x n), r = A^T b; 32x32 tiles, 256 threads (each 4 outputs)
__global__ void k_kappa_normal(int rows, int n, const double *A, const double *b, double *M, double *r)
{
    __shared__ double ta[32][33], tb[32][33];
    int i0 = blockIdx.y * 32, j0 = blockIdx.x * 32;
    int tx = threadIdx.x & 31, ty = threadIdx.x >> 5;  // ty in 0..7
    double acc[4] = {0, 0, 0, 0};
    for (int m0 = 0; m0 < rows; m0 += 32) {
        for (int q = 0; q < 4; ++q) {
            int mm = m0 + ty + 8 * q;
            ta[ty + 8 * q][tx] = (mm < rows && i0 + tx < n) ? A[(size_t)mm * n + i0 + tx] : 0.0;
            tb[ty + 8 * q][tx] = (mm < rows && j0 + tx < n) ? A[(size_t)mm * n + j0 + tx] : 0.0;
        }
        __syncthreads();
        for (int mm = 0; mm < 32; ++mm)
            for (int q = 0; q < 4; ++q) acc[q] += ta[mm][ty + 8 * q] * tb[mm][tx];
        __syncthreads();
    }
    for (int q = 0; q < 4; ++q) {
        int i = i0 + ty + 8 * q, j = j0 + tx;
        if (i < n && j < n) M[(size_t)i * n + j] = acc[q];
    }
    if (blockIdx.x == 0) {
        // r = A^T b for rows i0..i0+31
        if (threadIdx.x < 32) {
            int i = i0 + threadIdx.x;
            if (i < n) {
                double s = 0.0;
                for (int mm = 0; mm < rows; ++mm) s += A[(size_t)mm * n + i] * b[mm];
                r[i] = s;
            }
        }
    }
}

// Blocked right-looking Cholesky of the lower triangle of M (n x n, row-major),
// panels of kCholNb columns: for each panel k0 the diagonal block is factored
// by one CTA (k_chol_diag), the rows below it are solved against that factor
// (k_chol_panel, L21 = A21 L11^-T, one CTA per kCholNb rows), and the trailing
// lower triangle is updated, A22 -= L21 L21^T, by one CTA per kCholNb x
// kCholNb tile (k_chol_update).  Same arithmetic as the unblocked
// factorisation up to the order of the sums; a non-positive pivot sets
// ERR_SOLVE (the solve then continues on a placeholder pivot).
constexpr int kCholNb = 32;

__global__ void k_chol_diag(int n, int k0, double *M, unsigned *err)
{
    __shared__ double a[kCholNb][kCholNb + 1];
    const int nb = min(kCholNb, n - k0);
    const int r = threadIdx.x / kCholNb, c = threadIdx.x % kCholNb;
    const bool in = r < nb && c < nb && c <= r;
    if (in) a[r][c] = M[(size_t)(k0 + r) * n + k0 + c];
    __syncthreads();
    for (int j = 0; j < nb; ++j) {
        if (r == j && c == j) {
            double v = a[j][j];
            if (!(v > 0.0)) { atomicOr(err, (unsigned)ERR_SOLVE); v = 1e-300; }
            a[j][j] = sqrt(v);
        }
        __syncthreads();
        if (in && c == j && r > j) a[r][j] /= a[j][j];
        __syncthreads();
        if (in && c > j) a[r][c] -= a[r][j] * a[c][j];
        __syncthreads();
    }
    if (in) M[(size_t)(k0 + r) * n + k0 + c] = a[r][c];
}

// rows r0 = k0 + nb + blockIdx.x kCholNb .. (+kCholNb) of the panel: X L11^T = A21
__global__ void k_chol_panel(int n, int k0, double *M)
{
    __shared__ double L[kCholNb][kCholNb + 1], X[kCholNb][kCholNb + 1];
    const int nb = min(kCholNb, n - k0);
    const int r0 = k0 + nb + blockIdx.x * kCholNb;
    const int r = threadIdx.x / kCholNb, c = threadIdx.x % kCholNb;
    const bool row_in = r0 + r < n && c < nb;
    L[r][c] = (r < nb && c <= r) ? M[(size_t)(k0 + r) * n + k0 + c] : 0.0;
    X[r][c] = row_in ? M[(size_t)(r0 + r) * n + k0 + c] : 0.0;
    __syncthreads();
    for (int j = 0; j < nb; ++j) {
        if (c == j) X[r][j] /= L[j][j];
        __syncthreads();
        if (c > j && c < nb) X[r][c] -= X[r][j] * L[c][j];
        __syncthreads();
    }
    if (row_in) M[(size_t)(r0 + r) * n + k0 + c] = X[r][c];
}

// trailing update of the lower triangle below the panel; blockIdx.x enumerates the
// tiles (ti >= tj) of the (n - k0 - nb)^2 trailing matrix in kCholNb blocks
__global__ void k_chol_update(int n, int k0, double *M)
{
    __shared__ double Li[kCholNb][kCholNb + 1], Lj[kCholNb][kCholNb + 1];
    const int nb = min(kCholNb, n - k0);
    const int t0 = k0 + nb;
    int t = blockIdx.x, ti = 0;
    while (t > ti) { t -= ti + 1; ++ti; }  // tile (ti, tj = t), tj <= ti
    const int tj = t;
    const int ri0 = t0 + ti * kCholNb, rj0 = t0 + tj * kCholNb;
    for (int e = threadIdx.x; e < kCholNb * kCholNb; e += blockDim.x) {
        const int a = e / kCholNb, q = e % kCholNb;
        Li[a][q] = (ri0 + a < n && q < nb) ? M[(size_t)(ri0 + a) * n + k0 + q] : 0.0;
        Lj[a][q] = (rj0 + a < n && q < nb) ? M[(size_t)(rj0 + a) * n + k0 + q] : 0.0;
    }
    __syncthreads();
    for (int e = threadIdx.x; e < kCholNb * kCholNb; e += blockDim.x) {
        const int a = e / kCholNb, b = e % kCholNb;
        const int row = ri0 + a, col = rj0 + b;
        if (row >= n || col > row) continue;
        double acc = 0.0;
        for (int q = 0; q < nb; ++q) acc += Li[a][q] * Lj[b][q];
        M[(size_t)row * n + col] -= acc;
    }
}

static void chol_blocked(int n, double *M, unsigned *err, cudaStream_t st)
{
    for (int k0 = 0; k0 < n; k0 += kCholNb) {
        const int nb = std::min(kCholNb, n - k0), rest = n - k0 - nb;
        k_chol_diag<<<1, kCholNb * kCholNb, 0, st>>>(n, k0, M, err);
        if (rest <= 0) break;
        const int nt = (rest + kCholNb - 1) / kCholNb;
        k_chol_panel<<<nt, kCholNb * kCholNb, 0, st>>>(n, k0, M);
        k_chol_update<<<nt * (nt + 1) / 2, 256, 0, st>>>(n, k0, M);
    }
}

// Solve L L^T x = r in place (x overwrites r); one CTA.
__global__ void k_kappa_trsv(int n, const double *M, double *r)
{
    __shared__ double xj;
    for (int j = 0; j < n; ++j) {  // forward: L y = r
        if (threadIdx.x == 0) { xj = r[j] / M[(size_t)j * n + j]; r[j] = xj; }
        __syncthreads();
        for (int i = j + 1 + threadIdx.x; i < n; i += blockDim.x) r[i] -= M[(size_t)i * n + j] * xj;
        __syncthreads();
    }
    for (int j = n - 1; j >= 0; --j) {  // backward: L^T x = y
        if (threadIdx.x == 0) { xj = r[j] / M[(size_t)j * n + j]; r[j] = xj; }
        __syncthreads();
        for (int i = threadIdx.x; i < j; i += blockDim.x) r[i] -= M[(size_t)j * n + i] * xj;
        __syncthreads();
    }
}

// Refinement of the least-squares solution (corrected semi-normal equations,
// Bjorck): s = b - A x, g = A^T s, solve L L^T d = g with the Cholesky factor
// already in M, x += d.  The normal equations alone leave an error of order
// cond(A)^2 eps; each refinement step brings it towards cond(A) eps, the
// accuracy of an orthogonal-factorisation solve.

// s[m] = b[m] - A[m,:] x; one warp per row
__global__ void k_kappa_resid(int rows, int n, const double *A, const double *b, const double *x, double *s)
{
    const int m = (blockIdx.x * blockDim.x + threadIdx.x) >> 5, lane = threadIdx.x & 31;
    if (m >= rows) return;
    const double *Ar = A + (size_t)m * n;
    double acc = 0.0;
    for (int i = lane; i < n; i += 32) acc += Ar[i] * x[i];
    for (int o = 16; o > 0; o >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, o);
    if (lane == 0) s[m] = b[m] - acc;
}

// g[i] = sum_m A[m,i] s[m]; one thread per column
__global__ void k_kappa_atv(int rows, int n, const double *A, const double *s, double *g)
{
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    double acc = 0.0;
    for (int m = 0; m < rows; ++m) acc += A[(size_t)m * n + i] * s[m];
    g[i] = acc;
}

__global__ void k_kappa_add(int n, double *x, const double *d)
{
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n) x[i] += d[i];
}

// ---------------------------------------------------------------------------
// Fourier-segment generator (Eq. 9): segments of n = 256 M steps per dof,
// eta_t = (1/sqrt(n)) sum_j c_j e^{+2 pi i j t/n}, c_0 = sqrt(S_0) xi_0,
// c_{n/2} = sqrt(S_{n/2}) xi_1, c_j = sqrt(S_j/2) (xi_2j + i xi_2j+1) and
// c_{n-j} = conj(c_j), xi the white stream of the dof over the segment.

// sqrt(S_j / n) on w_j = 2 pi j/(n dt), j = 0..n/2, per system
template <class R>
__global__ void k_spectrum_seg(const DSpec *spec, int n, R *sq)
{
    const DSpec sp = spec[blockIdx.y];
    const int j = blockIdx.x * blockDim.x + threadIdx.x;
    if (j > n / 2) return;
    sq[(size_t)blockIdx.y * (n / 2 + 1) + j] = (R)sqrt(spectrum_value(sp, 2.0 * kPi * j / (n * sp.dt)) / n);
}

constexpr int kSegPairs = 2;  // dof pairs per CTA of the segment generator

// One CTA per kSegPairs pairs of dofs of one system: the n normals of each dof
// (the white stream over the segment's steps), the spectrum W = Z_a + i Z_b of a
// pair (both Z Hermitian, so the inverse transform of W carries the two real
// sequences as its real and imaginary parts), a radix-2 Stockham inverse FFT
// in shared memory (ping-pong between two buffers), eta rows t = 0..n-1.
// Launched for every block; it generates only at the first block of a segment
// unless `force`.  grid = (ceil(max dofp / (2 kSegPairs)), nsys), 256 threads,
// dynamic smem 2 kSegPairs * 2 n * sizeof(R).
template <class R, class C>
__global__ void __launch_bounds__(256) k_fourier(Dev d, const R *sq, const R *tw, int n, int force)
{
    extern __shared__ __align__(16) unsigned char fsm[];
    const long long blk = d.clock[0];
    const int M = n / kBlockSteps;
    const long long seg = floor_div(blk, M);
    if (!force && blk != seg * M) return;
    const DSys S = d.sys[blockIdx.y];
    const int dof_first = blockIdx.x * 2 * kSegPairs;
    if (dof_first >= S.dofp) return;
    const int nreal = 3 * S.N * S.P, h = n / 2;
    const size_t span = (size_t)2 * n;  // one pair's complex sequence
    R *bufA = reinterpret_cast<R *>(fsm);
    R *bufB = bufA + kSegPairs * span;
    // 1) normals: pair p, dof a (0) or b (1), step t -> bufB[p span + ab n + t]
    const int nq = n / 4;
    for (int w = threadIdx.x; w < kSegPairs * 2 * nq; w += blockDim.x) {
        const int q = w % nq, ab = (w / nq) & 1, p = w / (2 * nq);
        const int dofl = dof_first + 2 * p + ab;
        C z0 = 0, z1 = 0, z2 = 0, z3 = 0;
        if (dofl < nreal) {
            const unsigned long long uq = (unsigned long long)(seg * nq + q);
            uint4 ctr = make_uint4((uint32_t)uq, (uint32_t)dofl, 0u, (uint32_t)(uq >> 32));
            uint4 r = philox4x32_10(ctr, (uint32_t)d.seed, (uint32_t)(d.seed >> 32) ^ (uint32_t)blockIdx.y);
            bm_pair(r.x, r.y, z0, z1);
            bm_pair(r.z, r.w, z2, z3);
        }
        R *dst = bufB + p * span + ab * n + 4 * q;
        dst[0] = (R)z0; dst[1] = (R)z1; dst[2] = (R)z2; dst[3] = (R)z3;
    }
    __syncthreads();
    // 2) W_j = Z_a,j + i Z_b,j (sq holds sqrt(S_j/n): the 1/sqrt(n) is folded in)
    const R *sqs = sq + (size_t)blockIdx.y * (h + 1);
    for (int w = threadIdx.x; w < kSegPairs * n; w += blockDim.x) {
        const int j = w % n, p = w / n;
        const R *xa = bufB + p * span, *xb = xa + n;
        R re, im;
        if (j == 0) {
            re = sqs[0] * xa[0]; im = sqs[0] * xb[0];
        } else if (j == h) {
            re = sqs[h] * xa[1]; im = sqs[h] * xb[1];
        } else {
            const int jj = j < h ? j : n - j;
            const R r = sqs[jj] * (R)0.70710678118654752440;
            const R ar = xa[2 * jj], ai = xa[2 * jj + 1], br = xb[2 * jj], bi = xb[2 * jj + 1];
            if (j < h) { re = r * (ar - bi); im = r * (ai + br); }  // r (a_re + i a_im) + i r (b_re + i b_im)
            else { re = r * (ar + bi); im = r * (br - ai); }        // the conjugates
        }
        bufA[p * span + 2 * j] = re;
        bufA[p * span + 2 * j + 1] = im;
    }
    __syncthreads();
    // 3) sum_j W_j e^{+2 pi i j t/n}: stage (l, m) maps x[k + jj m], x[k + jj m + l m] to
    //    y[k + 2 jj m] = sum, y[k + 2 jj m + m] = e^{+2 pi i jj m/n} (difference)
    R *x = bufA, *y = bufB;
    for (int l = h, m = 1; l >= 1; l >>= 1, m <<= 1) {
        for (int w = threadIdx.x; w < kSegPairs * h; w += blockDim.x) {
            const int b = w % h, p = w / h;
            const int jj = b / m, k = b - jj * m;
            const R wr = tw[2 * (jj * m)], wi = tw[2 * (jj * m) + 1];
            const R *xp = x + p * span;
            R *yp = y + p * span;
            const int i0 = k + jj * m, i1 = i0 + l * m, o0 = k + 2 * jj * m, o1 = o0 + m;
            const R c0r = xp[2 * i0], c0i = xp[2 * i0 + 1], c1r = xp[2 * i1], c1i = xp[2 * i1 + 1];
            const R dr = c0r - c1r, di = c0i - c1i;
            yp[2 * o0] = c0r + c1r;
            yp[2 * o0 + 1] = c0i + c1i;
            yp[2 * o1] = fma(wr, dr, -wi * di);
            yp[2 * o1 + 1] = fma(wr, di, wi * dr);
        }
        __syncthreads();
        R *t = x;
        x = y;
        y = t;
    }
    // 4) eta rows of the segment (padding dofs: 0)
    R *eta = reinterpret_cast<R *>(d.eta);
    for (int w = threadIdx.x; w < kSegPairs * 2 * n; w += blockDim.x) {
        const int ab = w % 2, t = (w / 2) % n, p = w / (2 * n);
        const int dofl = dof_first + 2 * p + ab;
        if (dofl >= S.dofp) continue;
        eta[(size_t)t * d.Dtot + S.dof0 + dofl] = (dofl < nreal) ? x[p * span + 2 * t + ab] : R(0);
    }
}

// ---------------------------------------------------------------------------
// launchers

void launch_white(const Dev &d, int filter_kind, int max_dofp, int nsys, long long blk, cudaStream_t st)
{
    dim3 grid((unsigned)(((long long)max_dofp * 64 + 255) / 256), (unsigned)nsys);
    if (filter_kind == FK_FP64)
        k_white<double, double><<<grid, 256, 0, st>>>(d, blk);
    else if (filter_kind == FK_FP32)
        k_white<float, float><<<grid, 256, 0, st>>>(d, blk);
    else
        k_white<__nv_bfloat16, float><<<grid, 256, 0, st>>>(d, blk);
}

void launch_filter_simt(const Dev &d, int filter_kind, int max_dofp, int nsys, int Kmax, cudaStream_t st)
{
    dim3 grid((unsigned)max_dofp, (unsigned)nsys);
    if (filter_kind == FK_FP64) {
        size_t sm = sizeof(double) * (kBlockSteps + 3 * Kmax + 1);
        k_filter_simt<double><<<grid, kBlockSteps, sm, st>>>(d);
    } else {
        size_t sm = sizeof(float) * (kBlockSteps + 3 * Kmax + 1);
        k_filter_simt<float><<<grid, kBlockSteps, sm, st>>>(d);
    }
}

cudaError_t filter_simt_prepare(int Kmax)
{
    size_t sm = sizeof(double) * (kBlockSteps + 3 * Kmax + 1);
    cudaError_t e = cudaFuncSetAttribute(k_filter_simt<double>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         (int)sm);
    if (e != cudaSuccess) return e;
    return cudaFuncSetAttribute(k_filter_simt<float>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                (int)(sm / 2 + 16));
}

void launch_spectrum_taps(const DSpec *spec, int nsys, int Kmax, double *S, double *h64, float *h32,
                          const float *mlp_w, cudaStream_t st)
{
    k_spectrum<<<dim3((Kmax + 1 + 255) / 256, nsys), 256, 0, st>>>(spec, S);
    if (mlp_w) launch_spectrum_mlp(spec, nsys, Kmax, S, mlp_w, st);
    k_taps<<<dim3((Kmax + 1 + 127) / 128, nsys), 128, 0, st>>>(spec, S, h64, h32);
}

void launch_kappa_solve(int P, int n, double ymax, double y0, double *A, double *b, double *M, double *r,
                        double *work, unsigned *err, cudaStream_t st)
{
    int rows = 2 * n - 1;
    cudaMemsetAsync(A, 0, sizeof(double) * (size_t)rows * n, st);
    k_kappa_rows<<<(rows + 127) / 128, 128, 0, st>>>(P, n, ymax, y0, A, b);
    k_kappa_normal<<<dim3((n + 31) / 32, (n + 31) / 32), 256, 0, st>>>(rows, n, A, b, M, r);
    chol_blocked(n, M, err, st);
    k_kappa_trsv<<<1, 1024, 0, st>>>(n, M, r);
    double *s = work, *g = work + rows;
    for (int it = 0; it < kKappaRefine; ++it) {
        k_kappa_resid<<<(rows * 32 + 255) / 256, 256, 0, st>>>(rows, n, A, b, r, s);
        k_kappa_atv<<<(n + 127) / 128, 128, 0, st>>>(rows, n, A, s, g);
        k_kappa_trsv<<<1, 1024, 0, st>>>(n, M, g);
        k_kappa_add<<<(n + 255) / 256, 256, 0, st>>>(n, r, g);
    }
}


size_t fourier_smem(int n, int fp64) { return (size_t)2 * kSegPairs * 2 * n * (fp64 ? 8 : 4); }

cudaError_t fourier_prepare(int n)
{
    cudaError_t e = cudaFuncSetAttribute(k_fourier<float, float>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         (int)fourier_smem(n, 0));
    if (e != cudaSuccess) return e;
    return cudaFuncSetAttribute(k_fourier<double, double>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                (int)fourier_smem(n, 1));
}

void launch_spectrum_seg(const DSpec *spec, int nsys, int n, void *sq, int fp64, cudaStream_t st)
{
    dim3 g((unsigned)((n / 2 + 1 + 255) / 256), (unsigned)nsys);
    if (fp64) k_spectrum_seg<double><<<g, 256, 0, st>>>(spec, n, reinterpret_cast<double *>(sq));
    else k_spectrum_seg<float><<<g, 256, 0, st>>>(spec, n, reinterpret_cast<float *>(sq));
}

void launch_fourier(const Dev &d, int fp64, int max_dofp, int nsys, const void *sq, const void *tw, int n, int force,
                    cudaStream_t st)
{
    dim3 g((unsigned)((max_dofp + 2 * kSegPairs - 1) / (2 * kSegPairs)), (unsigned)nsys);
    const size_t sm = fourier_smem(n, fp64);
    if (fp64)
        k_fourier<double, double><<<g, 256, sm, st>>>(d, reinterpret_cast<const double *>(sq),
                                                      reinterpret_cast<const double *>(tw), n, force);
    else
        k_fourier<float, float><<<g, 256, sm, st>>>(d, reinterpret_cast<const float *>(sq),
                                                    reinterpret_cast<const float *>(tw), n, force);
}

}  // namespace qtb
