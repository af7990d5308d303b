// kappa_static.cu -- the kappa_P solve for callers that cannot allocate device
// memory.
//
// qtb_kappa_solve() obtains its scratch (the collocation matrix, the normal
// matrix and its Cholesky factor) with cudaMalloc on every call.  Some callers
// cannot do that: processes whose device memory is entirely reserved by
// another allocator (a framework's caching pool that owns the whole device, an
// MPS client with a fixed memory limit), where a cudaMalloc fails or would
// evict the pool, and latency-critical loops that must not touch the
// allocator, whose calls can block and synchronise the device.
// qtb_kappa_solve_noalloc() runs the same kernels on a fixed-size scratch
// array that lives in this file as a static __device__ variable, so it
// performs no allocation of any kind.  Every call synchronises its stream
// before returning (the non-positive-pivot check reads the error word back).
#include <cstdio>
#include <mutex>

#include "qtb_dev.cuh"
#include "qtb_kernels.cuh"

namespace {

constexpr int kNoallocMaxN = 512;  // largest collocation grid served
constexpr size_t kRows = 2 * (size_t)kNoallocMaxN - 1;
// A (rows x n) + b (rows) + M (n x n) + r (n) + refinement work (rows + n) + one error word
constexpr size_t kScratchDoubles =
    kRows * kNoallocMaxN + kRows + (size_t)kNoallocMaxN * kNoallocMaxN + kNoallocMaxN + kRows + kNoallocMaxN + 1;

// 6.3 MB, held on every device that loads the library until the process exits.
static __device__ __align__(256) double g_kappa_scratch[kScratchDoubles];

std::mutex g_mutex;
void *g_scratch_addr[256] = {nullptr};  // device address of the array, per device

__global__ void k_theta_grid(int n, double ymax, double y0, double *F)
{
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    const double dts = asinh(ymax / y0) / (n - 1);
    const double x = y0 * sinh(i * dts);
    F[i] = (x < 1e-6) ? 1.0 + x * x / 12.0 : x * (0.5 + 1.0 / expm1(x));
}

int fail_noalloc(int code, const char *msg)
{
    char buf[256];
    snprintf(buf, sizeof buf, "qtb_kappa_solve_noalloc: %s", msg);
    return qtb::set_last_error(code, buf);  // message returned by qtb_last_error()
}

}  // namespace

extern "C" int qtb_kappa_solve_noalloc(int P, int n, double y_max, double y0, double *F_dev, void *stream)
{
    if (P < 1 || !(y_max > 0) || !(y0 > 0) || !F_dev) return fail_noalloc(QTB_ERR_ARG, "bad arguments");
    if (n < 8 || n > kNoallocMaxN) return fail_noalloc(QTB_ERR_ARG, "n must be in 8..512 (size of the static scratch)");
    cudaStream_t st = (cudaStream_t)stream;
    if (P == 1) {  // kappa_1 = theta: no solve, no scratch
        k_theta_grid<<<(n + 127) / 128, 128, 0, st>>>(n, y_max, y0, F_dev);
        if (cudaGetLastError() != cudaSuccess) return fail_noalloc(QTB_ERR_CUDA, "launch failed");
        if (cudaStreamSynchronize(st) != cudaSuccess)
            return fail_noalloc(QTB_ERR_CUDA, cudaGetErrorString(cudaGetLastError()));
        return QTB_OK;
    }
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= 256) return fail_noalloc(QTB_ERR_CUDA, "no current device");
    void *base = nullptr;
    {
        // first call on a device: look up the array's device address with that device current
        std::lock_guard<std::mutex> lock(g_mutex);
        if (!g_scratch_addr[dev]) {
            void *ptr = nullptr;
            if (cudaGetSymbolAddress(&ptr, g_kappa_scratch) != cudaSuccess || !ptr)
                return fail_noalloc(QTB_ERR_CUDA, "cudaGetSymbolAddress of the static scratch failed");
            g_scratch_addr[dev] = ptr;
        }
        base = g_scratch_addr[dev];
    }
    const int rows = 2 * n - 1;
    double *A = (double *)base;
    double *b = A + (size_t)rows * n;
    double *M = b + rows;
    double *r = M + (size_t)n * n;
    double *work = r + n;
    unsigned *err = (unsigned *)(work + rows + n);
    // the array keeps the previous call's contents: clear what must start at zero
    if (cudaMemsetAsync(err, 0, sizeof(unsigned), st) != cudaSuccess) return fail_noalloc(QTB_ERR_CUDA, "memset failed");
    qtb::launch_kappa_solve(P, n, y_max, y0, A, b, M, r, work, err, st);  // also zeroes A
    if (cudaMemcpyAsync(F_dev, r, sizeof(double) * n, cudaMemcpyDeviceToDevice, st) != cudaSuccess)
        return fail_noalloc(QTB_ERR_CUDA, "copy of the solution failed");
    unsigned e = 0;
    if (cudaMemcpyAsync(&e, err, sizeof e, cudaMemcpyDeviceToHost, st) != cudaSuccess ||
        cudaStreamSynchronize(st) != cudaSuccess)
        return fail_noalloc(QTB_ERR_CUDA, cudaGetErrorString(cudaGetLastError()));
    if (e) return fail_noalloc(QTB_ERR_SOLVE, "non-positive pivot");
    return QTB_OK;
}
