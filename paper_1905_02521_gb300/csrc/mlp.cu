// mlp.cu -- learned stand-in for the kappa_P solve of Eq. 10.
//
// A 2-64-64-1 SiLU network maps (y = beta hbar w, P) to kappa_P/theta =
// F_P(y)/f(y).  Inputs x1 = asinh(y)/asinh(1000), x2 = (ln P - ln 2)/(ln 32 - ln 2).
// It is trained on the GPU with this file's kernels (per-sample forward and
// backward passes of 64 samples per CTA, deterministic fixed-order reduction
// of the CTA gradients, Adam), on F_P produced by the FP64 least-squares solve
// (qtb_kappa_solve), which also judges the trained model: for every trained P
// the maximum deviation from the solver on held-out frequencies is stored, and
// P values whose deviation exceeds the tolerance keep using the solver.
// Flat parameter layout (4417 floats): W1[64][2], b1[64], W2[64][64], b2[64], W3[64], b3.
#include <cmath>
#include <cstdint>
#include <cstring>
#include <vector>

#include "qtb_dev.cuh"
#include "qtb_kernels.cuh"

namespace qtb {

constexpr int kH = 64;
constexpr int kNP = kH * 2 + kH + kH * kH + kH + kH + 1;  // 4417
constexpr int oW1 = 0, oB1 = oW1 + 2 * kH, oW2 = oB1 + kH, oB2 = oW2 + kH * kH, oW3 = oB2 + kH, oB3 = oW3 + kH;
constexpr int kSamplesPerCta = 64;

__host__ __device__ inline float mlp_x1(double y) { return (float)(asinh(y) / asinh(1000.0)); }
__host__ __device__ inline float mlp_x2(int P) { return (float)((log((double)P) - log(2.0)) / (log(32.0) - log(2.0))); }

__device__ __forceinline__ float silu(float z) { return z / (1.0f + expf(-z)); }
__device__ __forceinline__ float dsilu(float z)
{
    const float s = 1.0f / (1.0f + expf(-z));
    return s * (1.0f + z * (1.0f - s));
}

// forward pass of one sample with the weights in (shared or global) memory
__device__ float mlp_forward(const float *w, float x1, float x2)
{
    float h1[kH];
#pragma unroll 8
    for (int i = 0; i < kH; ++i) h1[i] = silu(w[oW1 + 2 * i] * x1 + w[oW1 + 2 * i + 1] * x2 + w[oB1 + i]);
    float out = w[oB3];
    for (int j = 0; j < kH; ++j) {
        float z = w[oB2 + j];
#pragma unroll 16
        for (int i = 0; i < kH; ++i) z += w[oW2 + j * kH + i] * h1[i];
        out += w[oW3 + j] * silu(z);
    }
    return out;
}

// One CTA = 64 samples (one per thread): forward, backward, and the CTA's
// gradient of sum_s scale (out_s - t_s)^2 into gpart[blockIdx.x][kNP].
__global__ void __launch_bounds__(kSamplesPerCta) k_mlp_grad(const float *__restrict__ w, const float2 *__restrict__ x,
                                                            const float *__restrict__ t, int n, float scale,
                                                            float *gpart, float *lpart)
{
    extern __shared__ float sm[];
    float *sw = sm;                        // kNP weights
    float *sH1 = sw + kNP + 3;             // [64][65] activations of layer 1
    float *sG1 = sH1 + 64 * 65;            // dsilu(z1)
    float *sH2 = sG1 + 64 * 65;            // activations of layer 2
    float *sD2 = sH2 + 64 * 65;            // dL/dz2
    float *sD1 = sD2 + 64 * 65;            // dL/dz1
    float *sX = sD1 + 64 * 65;             // [64][2]
    float *sD3 = sX + 128;                 // [64]
    const int s = threadIdx.x;
    const int gidx = blockIdx.x * kSamplesPerCta + s;
    for (int p = s; p < kNP; p += blockDim.x) sw[p] = w[p];
    __syncthreads();
    const bool valid = gidx < n;
    const float2 xs = valid ? x[gidx] : make_float2(0.f, 0.f);
    sX[2 * s] = xs.x;
    sX[2 * s + 1] = xs.y;
    for (int i = 0; i < kH; ++i) {
        const float z = sw[oW1 + 2 * i] * xs.x + sw[oW1 + 2 * i + 1] * xs.y + sw[oB1 + i];
        sH1[s * 65 + i] = silu(z);
        sG1[s * 65 + i] = dsilu(z);
    }
    float out = sw[oB3];
    for (int j = 0; j < kH; ++j) {
        float z = sw[oB2 + j];
        for (int i = 0; i < kH; ++i) z += sw[oW2 + j * kH + i] * sH1[s * 65 + i];
        const float h = silu(z);
        sH2[s * 65 + j] = h;
        sD2[s * 65 + j] = dsilu(z);  // temporarily dsilu(z2)
        out += sw[oW3 + j] * h;
    }
    const float r = valid ? out - t[gidx] : 0.0f;
    const float d3 = 2.0f * scale * r;
    sD3[s] = d3;
    for (int j = 0; j < kH; ++j) sD2[s * 65 + j] *= d3 * sw[oW3 + j];
    for (int i = 0; i < kH; ++i) {
        float a = 0.0f;
        for (int j = 0; j < kH; ++j) a += sD2[s * 65 + j] * sw[oW2 + j * kH + i];
        sD1[s * 65 + i] = a * sG1[s * 65 + i];
    }
    // loss partial (fixed-order tree)
    __shared__ float red[kSamplesPerCta];
    red[s] = scale * r * r;
    __syncthreads();
    for (int o = kSamplesPerCta / 2; o > 0; o >>= 1) {
        if (s < o) red[s] += red[s + o];
        __syncthreads();
    }
    if (s == 0) lpart[blockIdx.x] = red[0];
    // gradient partials: each thread owns parameters p = s, s + 64, ...
    float *g = gpart + (size_t)blockIdx.x * kNP;
    for (int p = s; p < kNP; p += blockDim.x) {
        float acc = 0.0f;
        if (p < oB1) {
            const int i = p >> 1, k = p & 1;
            for (int q = 0; q < kSamplesPerCta; ++q) acc += sD1[q * 65 + i] * sX[2 * q + k];
        } else if (p < oW2) {
            const int i = p - oB1;
            for (int q = 0; q < kSamplesPerCta; ++q) acc += sD1[q * 65 + i];
        } else if (p < oB2) {
            const int j = (p - oW2) / kH, i = (p - oW2) % kH;
            for (int q = 0; q < kSamplesPerCta; ++q) acc += sD2[q * 65 + j] * sH1[q * 65 + i];
        } else if (p < oW3) {
            const int j = p - oB2;
            for (int q = 0; q < kSamplesPerCta; ++q) acc += sD2[q * 65 + j];
        } else if (p < oB3) {
            const int j = p - oW3;
            for (int q = 0; q < kSamplesPerCta; ++q) acc += sD3[q] * sH2[q * 65 + j];
        } else {
            for (int q = 0; q < kSamplesPerCta; ++q) acc += sD3[q];
        }
        g[p] = acc;
    }
}

size_t mlp_grad_smem() { return sizeof(float) * (kNP + 3 + 5 * 64 * 65 + 128 + 64); }

struct AdamState {
    int iter;  // Adam step count so far
};

// Sum the CTA partials in fixed order; optionally take one Adam step.
// One thread per parameter.  lr_sched: lr0 * decay^(iter / iters)
__global__ void k_mlp_reduce_adam(const float *gpart, int nblk, float *w, float *m, float *v, float *gout,
                                  const float *lpart, float *loss_out, AdamState *st, float lr0, float decay,
                                  int iters, int update)
{
    const int p = blockIdx.x * blockDim.x + threadIdx.x;
    const int it = st->iter;
    if (p < kNP) {
        float g = 0.0f;
        for (int b = 0; b < nblk; ++b) g += gpart[(size_t)b * kNP + p];
        if (gout) gout[p] = g;
        if (update) {
            const float b1 = 0.9f, b2 = 0.999f, eps = 1e-8f;
            const float mm = b1 * m[p] + (1.0f - b1) * g;
            const float vv = b2 * v[p] + (1.0f - b2) * g * g;
            m[p] = mm;
            v[p] = vv;
            const float tt = (float)(it + 1);
            const float lr = lr0 * powf(decay, (float)it / (float)iters);
            const float mh = mm / (1.0f - powf(b1, tt)), vh = vv / (1.0f - powf(b2, tt));
            w[p] -= lr * mh / (sqrtf(vh) + eps);
        }
    }
    if (p == 0 && loss_out) {
        float l = 0.0f;
        for (int b = 0; b < nblk; ++b) l += lpart[b];
        *loss_out = l;
    }
}

__global__ void k_mlp_tick(AdamState *st) { st->iter += 1; }

// ratio kappa_P/theta at n points
__global__ void k_mlp_infer(const float *w, const float2 *x, int n, float *out)
{
    const int k = blockIdx.x * blockDim.x + threadIdx.x;
    if (k >= n) return;
    out[k] = mlp_forward(w, x[k].x, x[k].y);
}

// S_j = kT f(y_j) ratio(y_j, P) W(w_j) for the systems in the learned mode.
// grid = (ceil((Kmax+1)/128), nsys)
__global__ void k_spectrum_mlp(const DSpec *spec, double *S, const float *w)
{
    const DSpec sp = spec[blockIdx.y];
    if (sp.mode != QTB_NOISE_QTB_PIMD_MLP) return;
    const int j = blockIdx.x * blockDim.x + threadIdx.x;
    if (j > sp.K) return;
    const int L = 2 * sp.K + 1;
    const double om = 2.0 * kPi * j / (L * sp.dt);
    const double kT = kBoltz * sp.T;
    const double y = kHbar * om / kT;
    const double fy = (y < 1e-6) ? 1.0 + y * y / 12.0 : y * (0.5 + 1.0 / expm1(y));
    const double ratio = (double)mlp_forward(w, mlp_x1(y), mlp_x2(sp.P));
    double W = 1.0;
    if (sp.omega_max > 0.0) W = 1.0 / (1.0 + exp((om - sp.omega_max) / (sp.omega_max / 50.0)));
    S[sp.taps0 + j] = kT * fy * ratio * W;
}

void launch_spectrum_mlp(const DSpec *spec, int nsys, int Kmax, double *S, const float *w, cudaStream_t st)
{
    k_spectrum_mlp<<<dim3((Kmax + 1 + 127) / 128, nsys), 128, 0, st>>>(spec, S, w);
}

}  // namespace qtb

using namespace qtb;

namespace {

double fth_host(double x)
{
    x = std::fabs(x);
    if (x < 1e-6) return 1.0 + x * x / 12.0;
    return x * (0.5 + 1.0 / std::expm1(x));
}

// F_P at y from the collocation grid (same interpolation as the library's spectrum)
double kappa_eval_host(const std::vector<double> &F, int P, double y, double ymax, double y0)
{
    const int n = (int)F.size();
    if (y > ymax) return fth_host(std::sqrt((double)P) * y) / P + std::sqrt((double)P) / (2.0 * y);
    const double dts = std::asinh(ymax / y0) / (n - 1);
    int i = (int)(std::asinh(y / y0) / dts);
    if (i > n - 2) i = n - 2;
    const double ya = y0 * std::sinh(i * dts), yb = y0 * std::sinh((i + 1) * dts);
    const double lam = (y - ya) / (yb - ya);
    return F[i] * (1.0 - lam) + F[i + 1] * lam;
}

// portable uniform in [0,1) from a 64-bit LCG (parameter initialisation)
struct Lcg {
    uint64_t s;
    double next()
    {
        s = s * 6364136223846793005ULL + 1442695040888963407ULL;
        return (double)(s >> 11) * (1.0 / 9007199254740992.0);
    }
};

}  // namespace

struct qtb_kappa_model {
    float *w = nullptr, *m = nullptr, *v = nullptr;
    std::vector<int> Ps;
    std::vector<double> val_err;  // per trained P: max |ratio_model - ratio_solver| on held-out points
    double tol = 0.0;
    double train_ms = 0.0;
    float final_loss = 0.0f;
};

extern "C" {

int qtb_kappa_model_create(qtb_kappa_model **out, unsigned long long seed)
{
    if (!out) return qtb::set_last_error(QTB_ERR_ARG, "qtb_kappa_model_create: out is NULL");
    qtb_kappa_model *M = new qtb_kappa_model();
    std::vector<float> w(kNP, 0.0f);
    Lcg g{seed ? seed : 1ULL};
    auto unif = [&](double a) { return (float)((2.0 * g.next() - 1.0) * a); };
    for (int p = oW1; p < oB1; ++p) w[p] = unif(std::sqrt(6.0 / 2.0));
    for (int p = oW2; p < oB2; ++p) w[p] = unif(std::sqrt(6.0 / kH));
    for (int p = oW3; p < oB3; ++p) w[p] = unif(std::sqrt(6.0 / kH));
    w[oB3] = 0.7f;
    if (cudaMalloc(&M->w, sizeof(float) * kNP) != cudaSuccess || cudaMalloc(&M->m, sizeof(float) * kNP) != cudaSuccess ||
        cudaMalloc(&M->v, sizeof(float) * kNP) != cudaSuccess) {
        delete M;
        return qtb::set_last_error(QTB_ERR_OOM, "qtb_kappa_model_create: device allocation failed");
    }
    cudaMemcpy(M->w, w.data(), sizeof(float) * kNP, cudaMemcpyHostToDevice);
    cudaMemset(M->m, 0, sizeof(float) * kNP);
    cudaMemset(M->v, 0, sizeof(float) * kNP);
    *out = M;
    return QTB_OK;
}

void qtb_kappa_model_destroy(qtb_kappa_model *M)
{
    if (!M) return;
    cudaFree(M->w);
    cudaFree(M->m);
    cudaFree(M->v);
    delete M;
}

int qtb_kappa_model_get_weights(qtb_kappa_model *M, float *w, int n)
{
    if (!M || !w || n < kNP) return qtb::set_last_error(QTB_ERR_ARG, "qtb_kappa_model_get_weights: need 4417 floats");
    return cudaMemcpy(w, M->w, sizeof(float) * kNP, cudaMemcpyDeviceToHost) == cudaSuccess
               ? QTB_OK : qtb::set_last_error(QTB_ERR_CUDA, "copy failed");
}

int qtb_kappa_model_set_weights(qtb_kappa_model *M, const float *w, int n)
{
    if (!M || !w || n < kNP) return qtb::set_last_error(QTB_ERR_ARG, "qtb_kappa_model_set_weights: need 4417 floats");
    return cudaMemcpy(M->w, w, sizeof(float) * kNP, cudaMemcpyHostToDevice) == cudaSuccess
               ? QTB_OK : qtb::set_last_error(QTB_ERR_CUDA, "copy failed");
}

// loss and gradient of the mean squared error over n samples (no update)
int qtb_kappa_model_grad(qtb_kappa_model *M, const float *x, const float *t, int n, float *grad, float *loss)
{
    if (!M || !x || !t || !grad || n < 1) return qtb::set_last_error(QTB_ERR_ARG, "qtb_kappa_model_grad: bad arguments");
    const int nblk = (n + kSamplesPerCta - 1) / kSamplesPerCta;
    float *dx = nullptr, *dt = nullptr, *gp = nullptr, *lp = nullptr, *gd = nullptr, *ld = nullptr;
    AdamState *st = nullptr;
    cudaMalloc(&dx, sizeof(float) * 2 * n);
    cudaMalloc(&dt, sizeof(float) * n);
    cudaMalloc(&gp, sizeof(float) * (size_t)nblk * kNP);
    cudaMalloc(&lp, sizeof(float) * nblk);
    cudaMalloc(&gd, sizeof(float) * kNP);
    cudaMalloc(&ld, sizeof(float));
    cudaMalloc(&st, sizeof(AdamState));
    cudaMemset(st, 0, sizeof(AdamState));
    cudaMemcpy(dx, x, sizeof(float) * 2 * n, cudaMemcpyHostToDevice);
    cudaMemcpy(dt, t, sizeof(float) * n, cudaMemcpyHostToDevice);
    cudaFuncSetAttribute(k_mlp_grad, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)mlp_grad_smem());
    k_mlp_grad<<<nblk, kSamplesPerCta, mlp_grad_smem()>>>(M->w, reinterpret_cast<const float2 *>(dx), dt, n,
                                                          1.0f / n, gp, lp);
    k_mlp_reduce_adam<<<(kNP + 255) / 256, 256>>>(gp, nblk, M->w, M->m, M->v, gd, lp, ld, st, 0.f, 1.f, 1, 0);
    cudaError_t e = cudaGetLastError();
    if (e == cudaSuccess) e = cudaMemcpy(grad, gd, sizeof(float) * kNP, cudaMemcpyDeviceToHost);
    if (e == cudaSuccess && loss) e = cudaMemcpy(loss, ld, sizeof(float), cudaMemcpyDeviceToHost);
    cudaFree(dx); cudaFree(dt); cudaFree(gp); cudaFree(lp); cudaFree(gd); cudaFree(ld); cudaFree(st);
    return e == cudaSuccess ? QTB_OK : qtb::set_last_error(QTB_ERR_CUDA, cudaGetErrorString(e));
}

// Train on solver data for the bead counts P_list: per P, n_per_P samples with
// y uniform in asinh(y) on [0, asinh(1000)], targets F_P(y)/f(y) from the FP64
// solve; Adam on the full set for `iters` steps (lr decays 3e-3 -> 1e-5);
// the solver then judges the model on held-out points (val_err per P).
int qtb_kappa_model_train(qtb_kappa_model *M, const int *P_list, int nP, int n_per_P, int iters, double tol)
{
    if (!M || !P_list || nP < 1 || n_per_P < 16 || iters < 1) return qtb::set_last_error(QTB_ERR_ARG, "qtb_kappa_model_train: bad arguments");
    for (int k = 0; k < nP; ++k)
        if (P_list[k] < 2 || P_list[k] > 32) return qtb::set_last_error(QTB_ERR_ARG, "qtb_kappa_model_train: P must be in 2..32");
    const int ng = 1024;
    const double ymax = 1000.0, y0 = 1.0;
    const double U = std::asinh(ymax);
    std::vector<float> X, Tg, Xv, Tv;
    std::vector<std::vector<double>> Fs(nP);
    for (int k = 0; k < nP; ++k) {
        const int P = P_list[k];
        Fs[k].resize(ng);
        int rc = qtb_kappa_solve(P, ng, ymax, y0, Fs[k].data());
        if (rc) return rc;
        for (int i = 0; i < n_per_P; ++i) {
            const double y = std::sinh(U * (i + 0.5) / n_per_P);
            X.push_back(mlp_x1(y));
            X.push_back(mlp_x2(P));
            Tg.push_back((float)(kappa_eval_host(Fs[k], P, y, ymax, y0) / fth_host(std::sqrt(1.0) * y)));
        }
        for (int i = 0; i < n_per_P / 4; ++i) {  // held-out points between the training points
            const double y = std::sinh(U * (4 * i + 2.0) / n_per_P);
            Xv.push_back(mlp_x1(y));
            Xv.push_back(mlp_x2(P));
            Tv.push_back((float)(kappa_eval_host(Fs[k], P, y, ymax, y0) / fth_host(y)));
        }
    }
    const int n = (int)Tg.size(), nv = (int)Tv.size();
    const int nblk = (n + kSamplesPerCta - 1) / kSamplesPerCta;
    float *dx = nullptr, *dt = nullptr, *gp = nullptr, *lp = nullptr, *ld = nullptr, *dxv = nullptr, *dov = nullptr;
    AdamState *st = nullptr;
    cudaMalloc(&dx, sizeof(float) * 2 * n);
    cudaMalloc(&dt, sizeof(float) * n);
    cudaMalloc(&gp, sizeof(float) * (size_t)nblk * kNP);
    cudaMalloc(&lp, sizeof(float) * nblk);
    cudaMalloc(&ld, sizeof(float));
    cudaMalloc(&dxv, sizeof(float) * 2 * nv);
    cudaMalloc(&dov, sizeof(float) * nv);
    cudaMalloc(&st, sizeof(AdamState));
    cudaMemset(st, 0, sizeof(AdamState));
    cudaMemset(M->m, 0, sizeof(float) * kNP);
    cudaMemset(M->v, 0, sizeof(float) * kNP);
    cudaMemcpy(dx, X.data(), sizeof(float) * X.size(), cudaMemcpyHostToDevice);
    cudaMemcpy(dt, Tg.data(), sizeof(float) * Tg.size(), cudaMemcpyHostToDevice);
    cudaMemcpy(dxv, Xv.data(), sizeof(float) * Xv.size(), cudaMemcpyHostToDevice);
    cudaFuncSetAttribute(k_mlp_grad, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)mlp_grad_smem());
    cudaStream_t sm;
    cudaStreamCreateWithFlags(&sm, cudaStreamNonBlocking);
    cudaEvent_t e0, e1;
    cudaEventCreate(&e0);
    cudaEventCreate(&e1);
    // one CUDA graph of 50 Adam iterations, replayed
    const int per_graph = 50;
    cudaGraph_t g;
    cudaGraphExec_t ge = nullptr;
    cudaStreamBeginCapture(sm, cudaStreamCaptureModeThreadLocal);
    for (int it = 0; it < per_graph; ++it) {
        k_mlp_grad<<<nblk, kSamplesPerCta, mlp_grad_smem(), sm>>>(M->w, reinterpret_cast<const float2 *>(dx), dt, n,
                                                                  1.0f / n, gp, lp);
        k_mlp_reduce_adam<<<(kNP + 255) / 256, 256, 0, sm>>>(gp, nblk, M->w, M->m, M->v, nullptr, lp, ld, st, 3e-3f,
                                                             3e-3f, iters, 1);
        k_mlp_tick<<<1, 1, 0, sm>>>(st);
    }
    cudaError_t e = cudaStreamEndCapture(sm, &g);
    if (e == cudaSuccess) e = cudaGraphInstantiate(&ge, g, 0);
    if (e == cudaSuccess) {
        cudaGraphDestroy(g);
        cudaEventRecord(e0, sm);
        for (int done = 0; done < iters && e == cudaSuccess; done += per_graph) e = cudaGraphLaunch(ge, sm);
        cudaEventRecord(e1, sm);
        if (e == cudaSuccess) e = cudaStreamSynchronize(sm);
    }
    float ms = 0.f;
    if (e == cudaSuccess) {
        cudaEventElapsedTime(&ms, e0, e1);
        M->train_ms = ms;
        cudaMemcpy(&M->final_loss, ld, sizeof(float), cudaMemcpyDeviceToHost);
        k_mlp_infer<<<(nv + 127) / 128, 128>>>(M->w, reinterpret_cast<const float2 *>(dxv), nv, dov);
        std::vector<float> ov(nv);
        e = cudaMemcpy(ov.data(), dov, sizeof(float) * nv, cudaMemcpyDeviceToHost);
        M->Ps.assign(P_list, P_list + nP);
        M->val_err.assign(nP, 0.0);
        M->tol = tol;
        const int per = n_per_P / 4;
        for (int k = 0; k < nP; ++k)
            for (int i = 0; i < per; ++i)
                M->val_err[k] = std::max(M->val_err[k], (double)std::fabs(ov[k * per + i] - Tv[k * per + i]));
    }
    if (ge) cudaGraphExecDestroy(ge);
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    cudaStreamDestroy(sm);
    cudaFree(dx); cudaFree(dt); cudaFree(gp); cudaFree(lp); cudaFree(ld); cudaFree(dxv); cudaFree(dov); cudaFree(st);
    return e == cudaSuccess ? QTB_OK : qtb::set_last_error(QTB_ERR_CUDA, cudaGetErrorString(e));
}

// Training summary: per trained P (in the order given to the training call) the
// solver-judged maximum deviation of kappa_P/theta; plus training time and loss.
int qtb_kappa_model_info(qtb_kappa_model *M, int *P_out, double *err_out, int max, int *n_out, double *train_ms,
                         double *final_loss)
{
    if (!M || !n_out) return qtb::set_last_error(QTB_ERR_ARG, "qtb_kappa_model_info: bad arguments");
    const int n = std::min(max, (int)M->Ps.size());
    for (int k = 0; k < n; ++k) {
        if (P_out) P_out[k] = M->Ps[k];
        if (err_out) err_out[k] = M->val_err[k];
    }
    *n_out = n;
    if (train_ms) *train_ms = M->train_ms;
    if (final_loss) *final_loss = M->final_loss;
    return QTB_OK;
}

// ratio kappa_P/theta of the model at n points (host arrays)
int qtb_kappa_model_eval(qtb_kappa_model *M, int P, const double *y, int n, double *ratio)
{
    if (!M || !y || !ratio || n < 1) return qtb::set_last_error(QTB_ERR_ARG, "qtb_kappa_model_eval: bad arguments");
    std::vector<float> X(2 * (size_t)n);
    for (int k = 0; k < n; ++k) {
        X[2 * k] = mlp_x1(y[k]);
        X[2 * k + 1] = mlp_x2(P);
    }
    float *dx = nullptr, *dout = nullptr;
    cudaMalloc(&dx, sizeof(float) * 2 * n);
    cudaMalloc(&dout, sizeof(float) * n);
    cudaMemcpy(dx, X.data(), sizeof(float) * 2 * n, cudaMemcpyHostToDevice);
    k_mlp_infer<<<(n + 127) / 128, 128>>>(M->w, reinterpret_cast<const float2 *>(dx), n, dout);
    std::vector<float> o(n);
    cudaError_t e = cudaMemcpy(o.data(), dout, sizeof(float) * n, cudaMemcpyDeviceToHost);
    cudaFree(dx);
    cudaFree(dout);
    for (int k = 0; k < n; ++k) ratio[k] = o[k];
    return e == cudaSuccess ? QTB_OK : qtb::set_last_error(QTB_ERR_CUDA, cudaGetErrorString(e));
}

}  // extern "C"

namespace qtb {
// used by capi.cu: model weights (device) and whether P passed the solver's judgement
const float *kappa_model_weights(const qtb_kappa_model *M) { return M ? M->w : nullptr; }
bool kappa_model_accepts(const qtb_kappa_model *M, int P)
{
    if (!M) return false;
    for (size_t k = 0; k < M->Ps.size(); ++k)
        if (M->Ps[k] == P) return M->val_err[k] <= M->tol;
    return false;
}
}  // namespace qtb
