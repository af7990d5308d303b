// capi.cu -- host side of the C ABI declared in include/qtb.h.
//
// Owns the device layout of every system (bead-major SoA state, noise dofs
// padded to tensor-core tiles, cell and neighbour lists per bead replica), the
// noise pipeline (white blocks in a ring, coloured block per 256 steps) and the
// CUDA graph that replays one 256-step block; a neighbour-list rebuild, when a
// system requests one, runs inside that step's cooperative force launch.
#include <cuda.h>
#include <dlfcn.h>

#include <cmath>
#include <cstdarg>
#include <cstdio>
#include <cstring>
#include <map>
#include <string>
#include <vector>

#include "qtb_dev.cuh"
#include "qtb_kernels.cuh"

using namespace qtb;

namespace {

thread_local std::string g_err = "no error";

int fail(int code, const char *fmt, ...)
{
    char buf[512];
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(buf, sizeof buf, fmt, ap);
    va_end(ap);
    g_err = buf;
    return code;
}

#define CUDA_TRY(expr)                                                                      \
    do {                                                                                    \
        cudaError_t e_ = (expr);                                                            \
        if (e_ != cudaSuccess) return fail(QTB_ERR_CUDA, "%s: %s", #expr, cudaGetErrorString(e_)); \
    } while (0)

long long roundup(long long a, long long b) { return (a + b - 1) / b * b; }

struct HSys {
    int N, P, mode, n_taps;
    double omega_max, T, gamma, box[3];
};

}  // namespace

int qtb::set_last_error(int code, const char *msg)
{
    g_err = msg;
    return code;
}

struct qtb_ctx {
    cudaStream_t st = nullptr;
    double skin = 0.0;           // largest neighbour-list skin of the systems, A
    std::vector<double> skins;   // each system's skin, A
    qtb_params p{};
    std::vector<double> mass, charge, bA, brho, bC;
    bool mixed = false, pair = true;
    int fk = FK_FP64;  // ring / filter arithmetic
    size_t rsz = 8;    // sizeof(R)
    std::vector<HSys> hs;
    std::vector<DSys> ds;
    std::vector<DRep> dr;
    std::vector<int> cell_rep, icta_sys, lcta_rep, ccta_sys;
    Dev d{};
    MdLaunch ml{};
    PairTab tab{};
    PairTabT<float> tabf{};
    long long step = 0;
    long long dclock = 0;          // host mirror of the device clock
    bool stale = false;            // a state was set since the last force evaluation
    bool lists_built = false;      // the neighbour lists of every system exist
    unsigned *d_selftest = nullptr;  // [2] words of qtb_wait_selftest
    double *d_stage = nullptr;       // state upload staging: positions, velocities [P][N][3]
    size_t stage_n = 0;              // its size in doubles
    long long ring_hi = LLONG_MIN; // highest white block in the ring
    long long ring_lo = LLONG_MIN; // lowest white block in the ring
    long long eta_blk = LLONG_MIN; // block whose coloured noise is in eta
    // Fourier-segment generator (Eq. 9): segments of seg_blocks blocks
    int gen = QTB_GEN_FILTER, seg_blocks = 1;
    long long eta_seg = LLONG_MIN; // segment in eta
    void *d_sq = nullptr, *d_tw = nullptr;  // sqrt(S_j/n) per system, twiddles
    int Kmax = 0;
    int max_dofp = 0, max_repN = 0;
    size_t ring_bytes = 0;
    std::vector<void *> allocs;
    std::map<int, double *> kappaF;  // P -> device F grid
    double *dS = nullptr;            // spectrum scratch
    DSpec *dspec = nullptr;
    double *d_taps64 = nullptr;
    float *d_taps32 = nullptr;
    int taps_cap = 0;
    cudaGraphExec_t gexec = nullptr;
    bool graph_dirty = true;
    bool own_stream = false;
    // profiling (events recorded inside the captured block)
    bool profiling = false, capturing = false;
    std::vector<cudaEvent_t> ev;        // pairs: start, stop
    std::vector<int> ev_cls;            // class of each pair
    size_t ev_used = 0, ev_pairs = 0;
    bool prof_launched = false;
    // tensor-core filter
    CUtensorMap tmA, tmB;  // the type carries the alignment TMA descriptors need
    void *d_Bt = nullptr;
    size_t Bt_bytes = 0;
    int *d_tiles = nullptr;
    int n_tiles = 0;
    // learned kappa_P model (borrowed) and the source of each system's spectrum
    const qtb_kappa_model *kmodel = nullptr;
    std::vector<int> ksrc;  // 0: theta or white, 1: kappa_P solver, 2: learned model

    void *alloc(size_t bytes)
    {
        if (bytes == 0) bytes = 16;
        void *ptr = nullptr;
        if (p.dev_alloc) {
            ptr = p.dev_alloc(bytes, p.alloc_user);
        } else if (cudaMalloc(&ptr, bytes) != cudaSuccess) {
            ptr = nullptr;
        }
        if (ptr) allocs.push_back(ptr);
        return ptr;
    }
    void release(void *ptr)
    {
        if (!ptr) return;
        for (size_t i = 0; i < allocs.size(); ++i)
            if (allocs[i] == ptr) {
                allocs.erase(allocs.begin() + i);
                break;
            }
        if (p.dev_free) p.dev_free(ptr, p.alloc_user);
        else cudaFree(ptr);
    }
    ~qtb_ctx()
    {
        if (gexec) cudaGraphExecDestroy(gexec);
        if (st) cudaStreamSynchronize(st);
        else cudaDeviceSynchronize();
        for (void *ptr : allocs) {
            if (p.dev_free) p.dev_free(ptr, p.alloc_user);
            else cudaFree(ptr);
        }
        for (cudaEvent_t e : ev) cudaEventDestroy(e);
        if (own_stream) cudaStreamDestroy(st);
    }
};

namespace {

template <class T>
T *upload(qtb_ctx *c, const std::vector<T> &v)
{
    T *ptr = (T *)c->alloc(sizeof(T) * (v.empty() ? 1 : v.size()));
    if (ptr && !v.empty()) cudaMemcpyAsync(ptr, v.data(), sizeof(T) * v.size(), cudaMemcpyHostToDevice, c->st);
    return ptr;
}

// Normal-mode matrix of the cyclic ring polymer (real Fourier basis), C[b][k].
void nm_matrix(int P, std::vector<double> &C)
{
    C.assign((size_t)P * P, 0.0);
    for (int b = 0; b < P; ++b)
        for (int k = 0; k < P; ++k) {
            double v;
            const double ang = 2.0 * kPi * (double)((b * k) % P) / P;
            if (k == 0) v = 1.0 / std::sqrt((double)P);
            else if (2 * k < P) v = std::sqrt(2.0 / P) * std::cos(ang);
            else if (2 * k == P) v = ((b % 2) ? -1.0 : 1.0) / std::sqrt((double)P);
            else v = std::sqrt(2.0 / P) * std::sin(ang);
            C[(size_t)b * P + k] = v;
        }
}

// exp(x^2) erfc(x) on 0 <= x <= xmax as a degree-11 polynomial in
// u = 2 x / xmax - 1: Chebyshev interpolation at the 12 Chebyshev nodes
// (near-minimax, relative error ~4e-9), converted to monomial coefficients.
void fit_erfcx(double xmax, double c[12])
{
    const int n = 12;
    for (int k = 0; k < n; ++k) c[k] = 0.0;
    if (!(xmax > 0.0)) {
        c[0] = 1.0;
        return;
    }
    double a[12];
    for (int k = 0; k < n; ++k) {
        double s = 0.0;
        for (int i = 0; i < n; ++i) {
            const double th = kPi * (i + 0.5) / n;
            const double x = (std::cos(th) + 1.0) * 0.5 * xmax;
            s += std::exp(x * x) * std::erfc(x) * std::cos(k * th);
        }
        a[k] = 2.0 * s / n;
    }
    a[0] *= 0.5;
    double Tm[12][12] = {{0}};  // monomial coefficients of the Chebyshev polynomials
    Tm[0][0] = 1.0;
    Tm[1][1] = 1.0;
    for (int k = 2; k < n; ++k)
        for (int j = 0; j < n; ++j) Tm[k][j] = (j > 0 ? 2.0 * Tm[k - 1][j - 1] : 0.0) - Tm[k - 2][j];
    for (int k = 0; k < n; ++k)
        for (int j = 0; j < n; ++j) c[j] += a[k] * Tm[k][j];
}

static int decode_err_word(qtb_ctx *c, unsigned e);

int check_err_word(qtb_ctx *c)
{
    unsigned e = 0;
    CUDA_TRY(cudaMemcpyAsync(&e, c->d.err, sizeof e, cudaMemcpyDeviceToHost, c->st));
    CUDA_TRY(cudaStreamSynchronize(c->st));
    return decode_err_word(c, e);
}

static int decode_err_word(qtb_ctx *c, unsigned e)
{
    if (e & ERR_OVERFLOW) return fail(QTB_ERR_OVERFLOW, "a cell-list cell exceeded its capacity (%d)", c->d.cap);
    if (e & ERR_NBR_OVERFLOW)
        return fail(QTB_ERR_OVERFLOW, "a neighbour list exceeded its capacity (%d entries)", c->d.maxnb);
    if (e & ERR_NONFINITE) return fail(QTB_ERR_NONFINITE, "non-finite energy: the integration blew up");
    if (e & ERR_SOLVE) return fail(QTB_ERR_SOLVE, "kappa_P solve: non-positive pivot");
    if (e & ERR_TIMEOUT_TC) return fail(QTB_ERR_TIMEOUT, "tensor-core filter: a bounded barrier wait gave up");
    if (e & ERR_TIMEOUT_BAR) return fail(QTB_ERR_TIMEOUT, "step kernel: a bounded grid-barrier wait gave up");
    if (e & ERR_CELL)
        return fail(QTB_ERR_STATE, "npt: the cell shrank below %.2f of its initial edges (the margin of its cell lists)",
                    kCellMinScale);
    return QTB_OK;
}

// ---- state transfer ------------------------------------------------------

int upload_state(qtb_ctx *c, int s, const double *pos, const double *vel)
{
    // one copy per array into a staging buffer, the conversion on the device
    // (k_load_state), one synchronisation: the caller's arrays are borrowed
    // for the call only (pinned host memory makes the copies plain DMA)
    if (!pos && !vel) return QTB_OK;
    const HSys &h = c->hs[s];
    const size_t n3 = 3 * (size_t)h.N * h.P;
    if (c->stage_n < 2 * n3) {
        c->d_stage = (double *)c->alloc(sizeof(double) * 2 * n3);  // freed with the context
        if (!c->d_stage) return fail(QTB_ERR_OOM, "device allocation failed");
        c->stage_n = 2 * n3;
    }
    double *dp = pos ? c->d_stage : nullptr, *dv = vel ? c->d_stage + n3 : nullptr;
    if (pos) CUDA_TRY(cudaMemcpyAsync(dp, pos, sizeof(double) * n3, cudaMemcpyHostToDevice, c->st));
    if (vel) CUDA_TRY(cudaMemcpyAsync(dv, vel, sizeof(double) * n3, cudaMemcpyHostToDevice, c->st));
    // once the lists exist, an uploaded position is stored as its periodic copy
    // nearest the reference of the last rebuild (positions are not wrapped between
    // rebuilds): an unchanged state then keeps its lists
    launch_load_state(c->d, c->ml, s, (long long)n3, dp, dv, (c->pair && c->lists_built) ? 1 : 0, c->st);
    CUDA_TRY(cudaGetLastError());
    CUDA_TRY(cudaStreamSynchronize(c->st));
    return QTB_OK;
}

// which: 0 positions, 1 velocities, 2 forces
int download(qtb_ctx *c, int s, int which, double *out)
{
    // converted on the device into the staging buffer, one copy, one synchronisation
    const HSys &h = c->hs[s];
    const size_t n3 = 3 * (size_t)h.N * h.P;
    if (c->stage_n < n3) {
        c->d_stage = (double *)c->alloc(sizeof(double) * 2 * n3);  // freed with the context
        if (!c->d_stage) return fail(QTB_ERR_OOM, "device allocation failed");
        c->stage_n = 2 * n3;
    }
    launch_store_state(c->d, c->ml, s, (long long)n3, which, c->d_stage, c->st);
    CUDA_TRY(cudaGetLastError());
    CUDA_TRY(cudaMemcpyAsync(out, c->d_stage, sizeof(double) * n3, cudaMemcpyDeviceToHost, c->st));
    CUDA_TRY(cudaStreamSynchronize(c->st));
    return QTB_OK;
}

// ---- pipeline pieces -------------------------------------------------------

void set_clock(qtb_ctx *c, long long b)
{
    if (c->dclock != b) {
        launch_setclock(c->d, b, c->st);
        c->dclock = b;
    }
}

// forces (and energies) at the current positions, the lists rebuilt where needed
// (all of them at the first evaluation); no velocity kick
int refresh_forces(qtb_ctx *c)
{
    set_clock(c, floor_div(c->step, kBlockSteps));
    const int j = (int)(c->step - c->dclock * kBlockSteps) - 1;
    const int cur = (int)(c->step & 1);  // positions of step s live in pos[s & 1]
    if (c->pair) {
        CUDA_TRY(cudaMemsetAsync(c->d.flag, 0, 2 * sizeof(unsigned), c->st));
        CUDA_TRY(cudaMemsetAsync(c->d.rflag, 0, 2 * sizeof(unsigned) * c->d.nsys, c->st));
        if (!c->lists_built) {
            // the first evaluation builds every system's lists (a nonzero word per system)
            CUDA_TRY(cudaMemsetAsync(c->d.flag + cur, 1, 1, c->st));
            CUDA_TRY(cudaMemsetAsync(c->d.rflag + (size_t)cur * c->d.nsys, 1, sizeof(unsigned) * c->d.nsys, c->st));
            c->lists_built = true;
        } else {
            // later ones (uploaded states) rebuild only the systems whose bead-atoms left
            // the skin/2 sphere around their positions at the last rebuild
            launch_refresh_check(c->d, c->ml, cur, c->st);
        }
    }
    launch_spring(c->d, c->ml, c->st);  // the record's spring term (no integrator ran)
    CUDA_TRY(launch_force(c->d, c->ml, c->tabf, c->tab, 0, j, cur, 0, 1, c->st));
    if (!c->pair) launch_reduce(c->d, c->ml, j, -1, c->st);  // the list force kernel reduces itself
    launch_centroid(c->d, c->ml, j, -1, 0, c->st);
    CUDA_TRY(cudaGetLastError());
    return QTB_OK;
}

void gen_white(qtb_ctx *c, long long blk)
{
    launch_white(c->d, c->fk, c->max_dofp, c->d.nsys, blk, c->st);
}

void filter_block(qtb_ctx *c)
{
    if (c->fk == FK_BF16)
        launch_filter_tc(c->d, &c->tmA, &c->tmB, c->n_tiles, c->d_tiles, c->st);
    else
        launch_filter_simt(c->d, c->fk, c->max_dofp, c->d.nsys, c->Kmax, c->st);
}

// cuTensorMapEncodeTiled from the driver library, resolved at run time so that
// the shared library loads on machines without a driver.
typedef CUresult (*EncodeTiledFn)(CUtensorMap *, CUtensorMapDataType, cuuint32_t, void *, const cuuint64_t *,
                                  const cuuint64_t *, const cuuint32_t *, const cuuint32_t *, CUtensorMapInterleave,
                                  CUtensorMapSwizzle, CUtensorMapL2promotion, CUtensorMapFloatOOBfill);

EncodeTiledFn encode_fn()
{
    static EncodeTiledFn fn = nullptr;
    if (!fn) {
        void *h = dlopen("libcuda.so.1", RTLD_NOW | RTLD_GLOBAL);
        if (h) fn = (EncodeTiledFn)dlsym(h, "cuTensorMapEncodeTiled");
    }
    return fn;
}

// Tensor-core filter set-up: Toeplitz band (BF16) of every system's taps,
// TMA descriptors of the white-noise ring (A) and of the band (B), tile table.
int setup_tc(qtb_ctx *c)
{
    EncodeTiledFn enc = encode_fn();
    if (!enc) return fail(QTB_ERR_CUDA, "cuTensorMapEncodeTiled not available (libcuda.so.1)");
    const int ns = (int)c->hs.size();
    const int Ktot = kBlockSteps * c->d.nslots, Ke = kBlockSteps * c->d.Kb;
    const size_t need = (size_t)ns * 256 * Ktot * 2;
    if (need > c->Bt_bytes) {
        c->release(c->d_Bt);
        c->d_Bt = c->alloc(need);
        if (!c->d_Bt) return fail(QTB_ERR_OOM, "Toeplitz band allocation failed");
        c->Bt_bytes = need;
    }
    launch_build_toeplitz(c->d, c->d_Bt, Ktot, Ke, c->st);
    CUDA_TRY(cudaGetLastError());
    std::vector<int> tiles;
    for (int s = 0; s < ns; ++s)
        for (int m = 0; m < c->ds[s].dofp; m += 128) {
            tiles.push_back(s);
            tiles.push_back(m);
        }
    c->n_tiles = (int)tiles.size() / 2;
    c->release(c->d_tiles);
    c->d_tiles = upload(c, tiles);
    if (!c->d_tiles) return fail(QTB_ERR_OOM, "tile table allocation failed");
    {
        const cuuint64_t dims[3] = {(cuuint64_t)kBlockSteps, (cuuint64_t)c->d.Dtot, (cuuint64_t)c->d.nslots};
        const cuuint64_t strides[2] = {(cuuint64_t)kBlockSteps * 2, (cuuint64_t)c->d.Dtot * kBlockSteps * 2};
        const cuuint32_t box[3] = {64, 128, 1}, es[3] = {1, 1, 1};
        CUresult r = enc(&c->tmA, CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 3, c->d.ring, dims, strides, box, es,
                         CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_128B, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
                         CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
        if (r != CUDA_SUCCESS) return fail(QTB_ERR_CUDA, "tensor map (noise ring) encode failed: %d", (int)r);
    }
    {
        const cuuint64_t dims[3] = {(cuuint64_t)Ktot, 256, (cuuint64_t)ns};
        const cuuint64_t strides[2] = {(cuuint64_t)Ktot * 2, (cuuint64_t)256 * Ktot * 2};
        const cuuint32_t box[3] = {64, 256, 1}, es[3] = {1, 1, 1};
        CUresult r = enc(&c->tmB, CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 3, c->d_Bt, dims, strides, box, es,
                         CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_128B, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
                         CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
        if (r != CUDA_SUCCESS) return fail(QTB_ERR_CUDA, "tensor map (Toeplitz band) encode failed: %d", (int)r);
    }
    CUDA_TRY(filter_tc_prepare());
    return QTB_OK;
}

// make the ring hold white blocks lo .. hi (hi - lo < nslots)
void ensure_ring(qtb_ctx *c, long long lo, long long hi)
{
    long long from = lo;
    const bool have = (c->ring_hi != LLONG_MIN && c->ring_lo <= lo && c->ring_hi >= lo - 1);
    if (have) from = c->ring_hi + 1;
    for (long long blk = from; blk <= hi; ++blk) gen_white(c, blk);
    if (!have) c->ring_lo = lo;
    if (!have || hi > c->ring_hi) c->ring_hi = std::max(hi, have ? c->ring_hi : hi);
    c->ring_lo = std::max(c->ring_lo, c->ring_hi - c->d.nslots + 1);
}

// make eta hold block b (ring then holds blocks b-Kb .. b+Kb)
void ensure_eta(qtb_ctx *c, long long b)
{
    if (c->gen == QTB_GEN_FOURIER) {
        const long long seg = floor_div(b, c->seg_blocks);
        set_clock(c, b);
        if (c->eta_seg != seg) {
            launch_fourier(c->d, c->mixed ? 0 : 1, c->max_dofp, c->d.nsys, c->d_sq, c->d_tw,
                           kBlockSteps * c->seg_blocks, 1, c->st);
            c->eta_seg = seg;
        }
        c->eta_blk = b;
        return;
    }
    if (c->eta_blk == b) return;
    ensure_ring(c, b - c->d.Kb, b + c->d.Kb);
    set_clock(c, b);
    filter_block(c);
    c->eta_blk = b;
}

// Profiling: event pairs recorded around each kernel class inside the graph
// (external event-record nodes), so that the per-kernel device time of the
// last replayed block can be read back.
enum { KC_WHITE = 0, KC_FILTER = 1, KC_INTEGRATE = 2, KC_CELLS = 3, KC_FORCE = 4, KC_REDUCE = 5, KC_N = 6 };

struct ProfMark {
    qtb_ctx *c;
    int cls;
    bool on;
    ProfMark(qtb_ctx *c_, int cls_);
    ~ProfMark();
};

ProfMark::ProfMark(qtb_ctx *c_, int cls_) : c(c_), cls(cls_), on(c_->profiling && c_->capturing)
{
    if (!on) return;
    const size_t pair = c->ev_used / 2;
    if (c->ev_used + 2 > c->ev.size()) {
        cudaEvent_t a, b;
        cudaEventCreate(&a);
        cudaEventCreate(&b);
        c->ev.push_back(a);
        c->ev.push_back(b);
        c->ev_cls.push_back(cls);
    } else {
        c->ev_cls[pair] = cls;
    }
    cudaEventRecordWithFlags(c->ev[c->ev_used], c->st, cudaEventRecordExternal);
}

ProfMark::~ProfMark()
{
    if (!on) return;
    cudaEventRecordWithFlags(c->ev[c->ev_used + 1], c->st, cudaEventRecordExternal);
    c->ev_used += 2;
}

// Steps j0 .. j0+count-1 of the current block, captured (graph) or launched.
// Positions of step s are in pos[s & 1].  Unfused: integrate, force.  Fused
// (one-bead systems): integrate once, then one force launch per step, each but
// the last also doing the first half of the next step.  A list rebuild, when
// requested, runs inside the force launch.  Profiling samples every 64th step
// of a captured block (event nodes cost about a microsecond each, so they are
// not put on every launch).
int run_steps(qtb_ctx *c, int j0, int count, bool graph)
{
    const MdLaunch &m = c->ml;
    const int obs = c->p.obs_stride;
    for (int t = 0; t < count; ++t) {
        const int j = j0 + t, cur = j & 1;
        const bool keep = c->capturing;
        if (j % 64 != 0) c->capturing = false;
        // isothermal-isobaric cells: updated here before the first step of the call
        // (fused) or of every step; in fused steps the step kernel updates them for
        // the next step
        if (c->p.npt && (!m.fused || t == 0)) launch_cell(c->d, j, c->mixed, c->st);
        if (!m.fused || t == 0) {
            ProfMark pm(c, KC_INTEGRATE);
            launch_integrate(c->d, m, j, cur, c->st);
        }
        const int adv = (m.fused && t < count - 1) ? 1 : 0;
        // may this step be recorded? (inside the graph the block index is only known on the device);
        // the cells need every step's kinetic energy and virial
        int rec;
        if (graph) rec = (kBlockSteps % obs == 0) ? ((j + 1) % obs == 0) : 1;
        else rec = ((c->step + t + 1) % obs == 0) ? 1 : 0;
        if (c->p.npt) rec = 1;
        {
            ProfMark pm(c, KC_FORCE);
            CUDA_TRY(launch_force(c->d, m, c->tabf, c->tab, 1, j, cur, adv, rec, c->st));
        }
        if (!m.pair || (rec && m.n_ccta)) {
            ProfMark pm(c, KC_REDUCE);
            if (!m.pair) launch_reduce(c->d, m, j, 1, c->st);
            if (rec) launch_centroid(c->d, m, j, 1, 1, c->st);
        }
        c->capturing = keep;
    }
    return QTB_OK;
}

int capture_block(qtb_ctx *c, cudaGraph_t *g)
{
    CUDA_TRY(cudaStreamBeginCapture(c->st, cudaStreamCaptureModeThreadLocal));
    c->capturing = true;
    c->ev_used = 0;
    int rc;
    if (c->gen == QTB_GEN_FOURIER) {
        // a new segment at the first block of each segment (the kernel tests the block clock)
        ProfMark m(c, KC_FILTER);
        launch_fourier(c->d, c->mixed ? 0 : 1, c->max_dofp, c->d.nsys, c->d_sq, c->d_tw,
                       kBlockSteps * c->seg_blocks, 0, c->st);
    } else {
        { ProfMark m(c, KC_WHITE); gen_white(c, LLONG_MIN); }  // block clock + Kb
        { ProfMark m(c, KC_FILTER); filter_block(c); }
    }
    rc = run_steps(c, 0, kBlockSteps, true);
    launch_tick(c->d, c->st);
    c->capturing = false;
    c->ev_pairs = c->ev_used / 2;
    cudaError_t e = cudaStreamEndCapture(c->st, g);
    if (rc) return rc;
    if (e != cudaSuccess) return fail(QTB_ERR_CUDA, "graph capture: %s", cudaGetErrorString(e));
    return QTB_OK;
}

int build_graph(qtb_ctx *c)
{
    if (c->gexec) {
        cudaGraphExecDestroy(c->gexec);
        c->gexec = nullptr;
    }
    cudaGraph_t g = nullptr;
    int rc = capture_block(c, &g);
    cudaError_t e = cudaSuccess;
    if (rc == QTB_OK) {
        e = cudaGraphInstantiate(&c->gexec, g, 0);
        cudaGraphDestroy(g);
    }
    if (rc) return rc;
    if (e != cudaSuccess) return fail(QTB_ERR_CUDA, "graph instantiate: %s", cudaGetErrorString(e));
    c->graph_dirty = false;
    return QTB_OK;
}

int ensure_kappa(qtb_ctx *c, int P)
{
    if (c->kappaF.count(P)) return QTB_OK;
    const int n = 1024;
    const double ymax = 1000.0, y0 = 1.0;
    const int rows = 2 * n - 1;
    double *F = (double *)c->alloc(sizeof(double) * n);
    double *A = (double *)c->alloc(sizeof(double) * (size_t)rows * n);
    double *b = (double *)c->alloc(sizeof(double) * rows);
    double *M = (double *)c->alloc(sizeof(double) * (size_t)n * n);
    double *work = (double *)c->alloc(sizeof(double) * (size_t)(rows + n));
    if (!F || !A || !b || !M || !work) return fail(QTB_ERR_OOM, "kappa_P solve: device allocation failed");
    launch_kappa_solve(P, n, ymax, y0, A, b, M, F, work, c->d.err, c->st);
    CUDA_TRY(cudaGetLastError());
    int rc = check_err_word(c);
    c->release(A);
    c->release(b);
    c->release(M);
    c->release(work);
    if (rc) return rc;
    c->kappaF[P] = F;
    return QTB_OK;
}

// Fourier-segment generator: sqrt(S_j/n) of every system on the segment grid
// (spectra as for the filter) and the twiddles e^{+2 pi i k/n}, k < n/2
int setup_fourier(qtb_ctx *c, const std::vector<DSpec> &spec)
{
    const int n = kBlockSteps * c->seg_blocks, ns = (int)c->hs.size();
    for (int s = 0; s < ns; ++s)
        if (spec[s].mode == QTB_NOISE_QTB_PIMD_MLP)
            return fail(QTB_ERR_ARG, "system %d: the learned kappa_P mode needs the filter generator", s);
    const size_t rs = c->mixed ? 4 : 8;
    c->release(c->d_sq);
    c->release(c->d_tw);
    c->d_sq = c->alloc(rs * (size_t)ns * (n / 2 + 1));
    c->d_tw = c->alloc(rs * (size_t)n);
    if (!c->d_sq || !c->d_tw) return fail(QTB_ERR_OOM, "segment spectrum allocation failed");
    launch_spectrum_seg(c->dspec, ns, n, c->d_sq, c->mixed ? 0 : 1, c->st);
    std::vector<double> tw((size_t)n);
    for (int k = 0; k < n / 2; ++k) {
        tw[2 * k] = std::cos(2.0 * kPi * k / n);
        tw[2 * k + 1] = std::sin(2.0 * kPi * k / n);
    }
    if (c->mixed) {
        std::vector<float> tf(tw.begin(), tw.end());
        CUDA_TRY(cudaMemcpyAsync(c->d_tw, tf.data(), 4 * tf.size(), cudaMemcpyHostToDevice, c->st));
        CUDA_TRY(cudaStreamSynchronize(c->st));
    } else {
        CUDA_TRY(cudaMemcpyAsync(c->d_tw, tw.data(), 8 * tw.size(), cudaMemcpyHostToDevice, c->st));
        CUDA_TRY(cudaStreamSynchronize(c->st));
    }
    CUDA_TRY(fourier_prepare(n));
    CUDA_TRY(cudaGetLastError());
    return QTB_OK;
}

// (re)build taps of every system from hs[].mode/n_taps/omega_max
int rebuild_filters(qtb_ctx *c)
{
    const int ns = (int)c->hs.size();
    int tot = 0, Kmax = 0;
    std::vector<DSpec> spec(ns);
    for (int s = 0; s < ns; ++s) {
        const HSys &h = c->hs[s];
        int K = (h.mode == QTB_NOISE_WHITE) ? 0 : (h.n_taps - 1) / 2;
        c->ds[s].K = K;
        c->ds[s].taps0 = tot;
        tot += K + 1;
        Kmax = std::max(Kmax, K);
        DSpec &sp = spec[s];
        sp.mode = h.mode;
        sp.K = K;
        sp.taps0 = c->ds[s].taps0;
        sp.P = h.P;
        sp.dt = c->p.dt;
        sp.T = h.T;
        sp.omega_max = h.omega_max;
        sp.F = nullptr;
        sp.n = 1024;
        sp.ymax = 1000.0;
        sp.y0 = 1.0;
        c->ksrc[s] = (h.mode == QTB_NOISE_QTB_PIMD) ? 1 : 0;
        if (h.mode == QTB_NOISE_QTB_PIMD_MLP) {
            // the learned model where the solver judged it within tolerance, else the solver
            if (h.P >= 2 && kappa_model_accepts(c->kmodel, h.P)) {
                c->ksrc[s] = 2;
            } else {
                sp.mode = QTB_NOISE_QTB_PIMD;
                c->ksrc[s] = 1;
            }
        }
        if (sp.mode == QTB_NOISE_QTB_PIMD) {
            int rc = ensure_kappa(c, h.P);
            if (rc) return rc;
            sp.F = c->kappaF[h.P];
        }
    }
    if (tot > c->taps_cap) {
        c->release(c->d_taps64);
        c->release(c->d_taps32);
        c->release(c->dS);
        c->d_taps64 = (double *)c->alloc(sizeof(double) * tot);
        c->d_taps32 = (float *)c->alloc(sizeof(float) * tot);
        c->dS = (double *)c->alloc(sizeof(double) * tot);
        if (!c->d_taps64 || !c->d_taps32 || !c->dS) return fail(QTB_ERR_OOM, "taps allocation failed");
        c->taps_cap = tot;
    }
    CUDA_TRY(cudaMemcpyAsync(c->dspec, spec.data(), sizeof(DSpec) * ns, cudaMemcpyHostToDevice, c->st));
    launch_spectrum_taps(c->dspec, ns, Kmax, c->dS, c->d_taps64, c->d_taps32, kappa_model_weights(c->kmodel), c->st);
    CUDA_TRY(cudaGetLastError());
    // ring geometry
    const int Kb = (Kmax + kBlockSteps - 1) / kBlockSteps;
    const int nslots = 2 * Kb + 1;
    const size_t esz = (c->fk == FK_FP64) ? 8 : (c->fk == FK_FP32 ? 4 : 2);
    const size_t need = esz * (size_t)nslots * (size_t)c->d.Dtot * kBlockSteps;
    if (need > c->ring_bytes || nslots != c->d.nslots) {
        if (need > c->ring_bytes) {
            c->release(c->d.ring);
            c->d.ring = c->alloc(need);
            if (!c->d.ring) return fail(QTB_ERR_OOM, "noise ring allocation (%zu bytes) failed", need);
            c->ring_bytes = need;
        }
        c->ring_hi = c->ring_lo = LLONG_MIN;
    }
    c->d.Kb = Kb;
    c->d.nslots = nslots;
    c->Kmax = Kmax;
    CUDA_TRY(filter_simt_prepare(Kmax));
    c->d.taps64 = c->d_taps64;
    c->d.tapsR = (c->fk == FK_FP64) ? (const void *)c->d_taps64 : (const void *)c->d_taps32;
    CUDA_TRY(cudaMemcpyAsync((void *)c->d.sys, c->ds.data(), sizeof(DSys) * ns, cudaMemcpyHostToDevice, c->st));
    if (c->fk == FK_BF16) {
        int rc = setup_tc(c);
        if (rc) return rc;
    }
    if (c->gen == QTB_GEN_FOURIER) {
        int rc = setup_fourier(c, spec);
        if (rc) return rc;
    }
    c->eta_blk = LLONG_MIN;
    c->eta_seg = LLONG_MIN;
    c->graph_dirty = true;
    return QTB_OK;
}

// skin of system s's neighbour lists: a given skin (> 0) for every system, none
// (< 0), or (0) min(r_cut/4, 0.8 A max(1, sqrt(T/300 K))): the thermal
// excursions that decide the rebuild rate grow as sqrt(T), and a hot system of a
// batch would otherwise rebuild on almost every step
double effective_skin(const qtb_params *p, double T)
{
    if (p->skin == 0.0) return std::min(0.25 * p->r_cut, 0.8 * std::max(1.0, std::sqrt(T / 300.0)));
    return p->skin < 0.0 ? 0.0 : p->skin;
}

int validate(const qtb_system *sys, int n_sys, const qtb_params *p)
{
    if (!sys || n_sys < 1 || !p) return fail(QTB_ERR_ARG, "qtb_init: need n_sys >= 1 systems and params");
    if (p->n_types < 1 || p->n_types > kMaxTypes) return fail(QTB_ERR_ARG, "n_types must be 1..%d", kMaxTypes);
    if (!p->mass) return fail(QTB_ERR_ARG, "mass table missing");
    if (!(p->dt > 0)) return fail(QTB_ERR_ARG, "dt must be > 0");
    if (p->potential < 0 || p->potential > 2) return fail(QTB_ERR_ARG, "unknown potential %d", p->potential);
    if (p->precision != QTB_FP64 && p->precision != QTB_MIXED) return fail(QTB_ERR_ARG, "unknown precision");
    if (p->filter_prec < 0 || p->filter_prec > 2) return fail(QTB_ERR_ARG, "unknown filter precision");
    if (p->obs_stride < 1 || p->max_records < 1) return fail(QTB_ERR_ARG, "obs_stride and max_records must be >= 1");
    if (p->nm_layout < 0 || p->nm_layout > 2) return fail(QTB_ERR_ARG, "nm_layout must be 0, 1 or 2");
    if (p->list_lanes != 0 && p->list_lanes != 8 && p->list_lanes != 16 && p->list_lanes != 32)
        return fail(QTB_ERR_ARG, "list_lanes must be 0, 8, 16 or 32");
    if (p->rebuild_scope != 0 && p->rebuild_scope != 1) return fail(QTB_ERR_ARG, "rebuild_scope must be 0 or 1");
    if (p->npt != 0 && p->npt != 1) return fail(QTB_ERR_ARG, "npt must be 0 or 1");
    if (p->npt) {
        if (p->potential != QTB_POT_PAIR) return fail(QTB_ERR_ARG, "npt: pair potential only");
        if (!(p->cell_mass > 0) || !(p->cell_gamma >= 0)) return fail(QTB_ERR_ARG, "npt: cell_mass > 0, cell_gamma >= 0");
        if (!std::isfinite(p->pressure)) return fail(QTB_ERR_ARG, "npt: pressure must be finite");
    }
    if (p->potential == QTB_POT_PAIR) {
        if (!p->charge || !p->buck_A || !p->buck_rho || !p->buck_C) return fail(QTB_ERR_ARG, "pair tables missing");
        if (!(p->r_cut > 0)) return fail(QTB_ERR_ARG, "r_cut must be > 0");
        if (!(effective_skin(p, 0.0) < 0.5 * p->r_cut)) return fail(QTB_ERR_ARG, "skin must be < r_cut/2");
    }
    for (int s = 0; s < n_sys; ++s) {
        const qtb_system &q = sys[s];
        if (q.n_atoms < 1 || q.n_beads < 1) return fail(QTB_ERR_ARG, "system %d: n_atoms, n_beads >= 1", s);
        if (q.n_atoms > (int)kNbIdx) return fail(QTB_ERR_ARG, "system %d: more than 2^26 - 1 atoms", s);
        if (!md_supported_P(q.n_beads)) return fail(QTB_ERR_ARG, "system %d: n_beads %d not supported (1-6, 8, 16, 32)", s, q.n_beads);
        if (!q.type || !q.pos) return fail(QTB_ERR_ARG, "system %d: type and pos required", s);
        if (!(q.T > 0) || !(q.gamma >= 0)) return fail(QTB_ERR_ARG, "system %d: T > 0, gamma >= 0", s);
        for (int i = 0; i < q.n_atoms; ++i)
            if (q.type[i] < 0 || q.type[i] >= p->n_types) return fail(QTB_ERR_ARG, "system %d: bad type at %d", s, i);
        if (p->potential == QTB_POT_PAIR)
            for (int c = 0; c < 3; ++c)
                if (!(q.box[c] >= p->r_cut)) return fail(QTB_ERR_ARG, "system %d: box edge %d must be >= r_cut", s, c);
    }
    return QTB_OK;
}

}  // namespace

// ===========================================================================

extern "C" {

const char *qtb_last_error(void) { return g_err.c_str(); }

int qtb_init(qtb_ctx **out, const qtb_system *sys, int n_sys, const qtb_params *p, void *stream)
{
    if (!out) return fail(QTB_ERR_ARG, "qtb_init: out is NULL");
    *out = nullptr;
    int rc = validate(sys, n_sys, p);
    if (rc) return rc;
    qtb_ctx *c = new qtb_ctx();
    c->st = (cudaStream_t)stream;
    if (!c->st) {
        // the legacy default stream cannot be captured into a graph: use our own
        if (cudaStreamCreateWithFlags(&c->st, cudaStreamNonBlocking) != cudaSuccess) {
            delete c;
            return fail(QTB_ERR_CUDA, "cudaStreamCreate failed");
        }
        c->own_stream = true;
    }
    c->p = *p;
    c->skins.resize(n_sys);
    c->skin = 0.0;  // the largest of the systems' skins
    for (int s = 0; s < n_sys; ++s) {
        c->skins[s] = effective_skin(p, sys[s].T);
        c->skin = std::max(c->skin, c->skins[s]);
    }
    const int nt = p->n_types;
    c->mass.assign(p->mass, p->mass + nt);
    c->mixed = (p->precision == QTB_MIXED);
    c->pair = (p->potential == QTB_POT_PAIR);
    c->fk = c->mixed ? (p->filter_prec == QTB_FILTER_BF16 ? FK_BF16 : FK_FP32) : FK_FP64;
    c->rsz = c->mixed ? 4 : 8;
    auto bail = [&](int code) {
        delete c;
        return code;
    };

    // ---- pair table (FP64 master, FP32 copy for the mixed kernels)
    PairTab &T = c->tab;
    memset(&T, 0, sizeof T);
    T.ntypes = nt;
    T.potential = p->potential;
    T.ext_V0 = p->ext_V0;
    T.ext_ia2 = 1.0 / (p->ext_a * p->ext_a);
    for (int a = 0; a < nt; ++a) {
        T.mass[a] = p->mass[a];
        T.mass_mvv[a] = p->mass[a] * kMvv2e;
        const float mh = (float)p->mass[a], kh = (float)(0.5 * p->mass[a] * kMvv2e);
        T.mass_ff[a] = make_float2(mh, (float)(p->mass[a] - (double)mh));
        T.half_mvv_ff[a] = make_float2(kh, (float)(0.5 * p->mass[a] * kMvv2e - (double)kh));
        T.hdt_m[a] = 0.5 * p->dt / (p->mass[a] * kMvv2e);
        T.ext_k[a] = p->mass[a] * kMvv2e * p->ext_omega * p->ext_omega;
    }
    if (c->pair) {
        const double rc_ = p->r_cut, al = p->dsf_alpha;
        T.rc = rc_;
        T.rc2 = rc_ * rc_;
        T.alpha = al;
        T.alpha2 = al * al;
        T.two_a_sqrtpi = 2.0 * al / std::sqrt(kPi);
        T.erfc_rc_over_rc = std::erfc(al * rc_) / rc_;
        T.rl2 = (rc_ + c->skin) * (rc_ + c->skin);
        T.fshift = std::erfc(al * rc_) / (rc_ * rc_) + 2.0 * al / std::sqrt(kPi) * std::exp(-al * al * rc_ * rc_) / rc_;
        for (int a = 0; a < nt; ++a)
            for (int b = 0; b < nt; ++b) {
                const int t = a * kMaxTypes + b, u = a * nt + b;
                T.A[t] = p->buck_A[u];
                T.inv_rho[t] = (p->buck_A[u] != 0.0) ? 1.0 / p->buck_rho[u] : 0.0;
                T.A_over_rho[t] = p->buck_A[u] * T.inv_rho[t];
                T.C[t] = p->buck_C[u];
                T.C6[t] = 6.0 * p->buck_C[u];
                T.qq[t] = kCoulomb * p->charge[a] * p->charge[b];
                double es = 0.0;
                if (p->buck_A[u] != 0.0) es += p->buck_A[u] * std::exp(-rc_ / p->buck_rho[u]);
                es -= p->buck_C[u] / std::pow(rc_, 6);
                T.eshift[t] = es;
            }
    }
    {
        PairTabT<float> &F = c->tabf;
        memset(&F, 0, sizeof F);
        const int NT = kMaxTypes * kMaxTypes;
        for (int t = 0; t < NT; ++t) {
            F.A[t] = (float)T.A[t]; F.inv_rho[t] = (float)T.inv_rho[t]; F.A_over_rho[t] = (float)T.A_over_rho[t];
            F.C[t] = (float)T.C[t]; F.C6[t] = (float)T.C6[t]; F.qq[t] = (float)T.qq[t]; F.eshift[t] = (float)T.eshift[t];
        }
        F.alpha = (float)T.alpha; F.alpha2 = (float)T.alpha2; F.two_a_sqrtpi = (float)T.two_a_sqrtpi;
        F.rc = (float)T.rc; F.rc2 = (float)T.rc2; F.erfc_rc_over_rc = (float)T.erfc_rc_over_rc; F.fshift = (float)T.fshift;
        for (int a = 0; a < kMaxTypes; ++a) {
            F.hdt_m[a] = (float)T.hdt_m[a]; F.ext_k[a] = (float)T.ext_k[a];
            F.mass[a] = T.mass[a]; F.mass_mvv[a] = T.mass_mvv[a];
            F.mass_ff[a] = T.mass_ff[a]; F.half_mvv_ff[a] = T.half_mvv_ff[a];
        }
        F.ext_V0 = (float)T.ext_V0; F.ext_ia2 = (float)T.ext_ia2;
        F.ntypes = T.ntypes; F.potential = T.potential;
        const double log2e = 1.4426950408889634;
        F.alpha2_l2e = (float)(T.alpha2 * log2e);
        F.rl2 = (float)T.rl2;
        const double xmax = T.alpha * T.rc;
        F.erfc_us = (xmax > 0.0) ? (float)(2.0 / xmax) : 0.0f;
        double cfit[12];
        fit_erfcx(xmax, cfit);
        for (int k = 0; k < 12; ++k) F.erfc_c[k] = (float)cfit[k];
    }

    // ---- layout
    long long G = 0, D = 0;
    int icta = 0, ccta = 0, nrep = 0, ncells = 0, cap = 8;
    int rot_tot = 0, nm_tot = 0;
    std::map<int, int> nm_off;
    std::vector<double> nmC_host;
    c->hs.resize(n_sys);
    c->ksrc.assign(n_sys, 0);
    c->ds.resize(n_sys);
    // Neighbour lists within r_list = r_cut + skin, built from cells >=
    // r_list/2 with a 5^3 stencil whose neighbourhood streams through shared
    // memory in chunks.
    // (each system's list radius r_cut + its skin; the pair table keeps the largest)
    auto r_list_of = [&](int s) { return p->r_cut + c->skins[s]; };
    auto cell_cap = [&](const qtb_system &q, double edge) {
        int nc[3];
        for (int k = 0; k < 3; ++k) nc[k] = std::max(1, (int)std::floor(q.box[k] / edge));
        const double e = (double)q.n_atoms / (nc[0] * nc[1] * nc[2]);
        int cp = (int)roundup((long long)std::ceil(1.25 * e + 4.0 * std::sqrt(e) + 8.0), 8);
        return std::min(cp, (int)roundup(q.n_atoms, 8));
    };
    // an isothermal-isobaric cell may shrink to kCellMinScale of its edges: the
    // cells (in the reference cell) and the lists keep that margin
    auto cell_edge_of = [&](int s) { return 0.5 * r_list_of(s) / (p->npt ? kCellMinScale : 1.0); };
    const double dens_margin = p->npt ? 1.0 / (kCellMinScale * kCellMinScale * kCellMinScale) : 1.0;
    int stage_cap = 0, maxnb = 32;
    if (c->pair) {
        double ecell = 0.0;
        for (int s = 0; s < n_sys; ++s) {
            const double r_list = r_list_of(s), cell_edge = cell_edge_of(s);
            const double vlist = 4.0 / 3.0 * kPi * r_list * r_list * r_list;
            int nc[3];
            for (int k = 0; k < 3; ++k) nc[k] = std::max(1, (int)std::floor(sys[s].box[k] / cell_edge));
            ecell = std::max(ecell, (double)sys[s].n_atoms / (nc[0] * nc[1] * nc[2]));
            // list capacity: 1.5 x the mean population of the list sphere plus a margin
            const double rho = sys[s].n_atoms / (sys[s].box[0] * sys[s].box[1] * sys[s].box[2]);
            maxnb = std::max(maxnb, (int)roundup((long long)std::ceil(1.5 * rho * dens_margin * vlist + 64.0), 32));
        }
        // staging chunk of the list build: 1.5 x the mean stencil population plus a
        // margin, between 512 entries (the sort keys share the buffer) and 1024
        // (the buffer is allocated for every CTA of the step kernel, a larger
        // neighbourhood takes several chunks)
        stage_cap = (int)std::max(512LL, std::min(roundup((long long)std::ceil(1.5 * kStencilCells * ecell) + 128, 64), 1024LL));
    }
    int nlcta = 0;
    // ring-polymer integrator layout: 32 atoms per CTA (coalesced rows) for large
    // contexts, fewer (more CTAs) for small ones
    long long beads_total = 0;
    for (int s = 0; s < n_sys; ++s) beads_total += (long long)sys[s].n_atoms * sys[s].n_beads;
    // bead-atom and dof indices are 32-bit on the device (3 dofs per bead-atom)
    if (beads_total > (long long)INT_MAX / 4)
        return bail(fail(QTB_ERR_ARG, "%lld bead-atoms in one context: at most %d", beads_total, INT_MAX / 4));
    const int nm_big = p->nm_layout == 2 ? 1 : p->nm_layout == 1 ? 0 : (beads_total >= (1LL << 18) ? 1 : 0);
    const int lanes = p->list_lanes ? p->list_lanes : 16;
    for (int s = 0; s < n_sys; ++s) {
        const qtb_system &q = sys[s];
        HSys &h = c->hs[s];
        h.N = q.n_atoms;
        h.P = q.n_beads;
        h.mode = QTB_NOISE_WHITE;
        h.n_taps = 1;
        h.omega_max = 0;
        h.T = q.T;
        h.gamma = q.gamma;
        for (int k = 0; k < 3; ++k) h.box[k] = q.box[k];
        DSys &S = c->ds[s];
        memset(&S, 0, sizeof S);
        S.N = h.N;
        S.P = h.P;
        S.g0 = (int)G;
        S.dof0 = (int)D;
        S.dofp = (int)roundup(3LL * h.N * h.P, kDofPad);
        G += (long long)h.N * h.P;
        D += S.dofp;
        S.icta0 = icta;
        icta += (h.N + integrate_atoms_per_cta(h.P, nm_big) - 1) / integrate_atoms_per_cta(h.P, nm_big);
        S.icta1 = icta;
        S.ccta0 = ccta;
        if (h.P > 1) ccta += (h.N + kCenAtoms - 1) / kCenAtoms;
        S.ccta1 = ccta;
        for (int k = 0; k < 3; ++k) S.box[k] = q.box[k];
        S.T = q.T;
        S.gamma = q.gamma;
        S.c1 = std::exp(-q.gamma * p->dt);
        S.wP = std::sqrt((double)h.P) * kBoltz * q.T / kHbar;
        S.invP = 1.0 / h.P;
        S.invP_f = (float)S.invP;
        S.c1_f = (float)S.c1;
        const double skin = c->skins[s];
        S.skin2 = 0.25 * skin * skin;
        S.skin2_f = (float)S.skin2;
        S.rl2 = (p->r_cut + skin) * (p->r_cut + skin);
        S.rl2_f = (float)S.rl2;
        {   // isothermal-isobaric: the particles' share of the skin (0.999: FP32 slack)
            const double tol = kNptCellSkin * skin / (p->r_cut + skin);
            const double D = 0.999 * 0.5 * (skin * (1.0 - tol) - tol * p->r_cut);
            S.npt_d2 = D * D;
            S.npt_d2_f = (float)S.npt_d2;
        }
        for (int k = 0; k < 3; ++k) {
            S.fix_scale[k] = (float)(q.box[k] / (double)(1 << kFixBits));
            S.fix_inv[k] = (q.box[k] > 0) ? (float)((double)(1 << kFixBits) / q.box[k]) : 0.f;
        }
        S.rot0 = rot_tot;
        rot_tot += h.P;
        if (!nm_off.count(h.P)) {
            std::vector<double> Cm;
            nm_matrix(h.P, Cm);
            nm_off[h.P] = nm_tot;
            nm_tot += h.P * h.P;
            nmC_host.insert(nmC_host.end(), Cm.begin(), Cm.end());
        }
        S.nm0 = nm_off[h.P];
        S.rep0 = nrep;
        S.cell0 = S.cell1 = ncells;
        c->max_dofp = std::max(c->max_dofp, S.dofp);
        if (c->pair) {
            int nc[3];
            for (int k = 0; k < 3; ++k) nc[k] = std::max(1, (int)std::floor(q.box[k] / cell_edge_of(s)));
            const int cells = nc[0] * nc[1] * nc[2];
            cap = std::max(cap, cell_cap(q, cell_edge_of(s)));
            for (int b = 0; b < h.P; ++b) {
                DRep R;
                memset(&R, 0, sizeof R);
                R.sys = s;
                R.g0 = S.g0 + b * h.N;
                R.N = h.N;
                for (int k = 0; k < 3; ++k) {
                    R.nc[k] = nc[k];
                    R.box[k] = q.box[k];
                    R.fix_scale[k] = S.fix_scale[k];
                }
                R.cell0 = ncells;
                ncells += cells;
                R.fcta0 = nlcta;
                const int nl = (h.N + list_atoms(lanes) - 1) / list_atoms(lanes);
                nlcta += nl;
                c->dr.push_back(R);
                for (int t = 0; t < cells; ++t) c->cell_rep.push_back(nrep);
                for (int t = 0; t < nl; ++t) c->lcta_rep.push_back(nrep);
                ++nrep;
            }
            S.cell1 = ncells;
        }
    }
    if (cap > kMaxCellCap)
        return bail(fail(QTB_ERR_ARG, "cell capacity %d > %d: box too dense for (r_cut + skin)/2 cells", cap, kMaxCellCap));
    for (int s = 0; s < n_sys; ++s)
        for (int t = c->ds[s].icta0; t < c->ds[s].icta1; ++t) c->icta_sys.push_back(s);
    for (int s = 0; s < n_sys; ++s)
        for (int t = c->ds[s].ccta0; t < c->ds[s].ccta1; ++t) c->ccta_sys.push_back(s);
    c->ml.mixed = c->mixed;
    c->ml.lanes = lanes;
    // minimum image suffices for the list entries when every edge exceeds twice the
    // largest separation an entry can reach before a rebuild (r_cut + skin, plus skin/2
    // of motion for each of the two atoms); not with a changing cell
    c->ml.minimg = (c->pair && c->mixed && !p->npt) ? 1 : 0;
    for (int s = 0; s < n_sys && c->ml.minimg; ++s)
        for (int k = 0; k < 3; ++k)
            if (!(sys[s].box[k] > 2.0 * (p->r_cut + 2.0 * c->skins[s]))) c->ml.minimg = 0;
    if (c->pair && step_prepare(c->ml, stage_cap) != cudaSuccess)
        return bail(fail(QTB_ERR_CUDA, "cannot prepare the cooperative step kernel (shared memory, occupancy)"));
    int ext_gx = 0;
    for (int s = 0; s < n_sys; ++s) ext_gx = std::max(ext_gx, (c->hs[s].N * c->hs[s].P + 127) / 128);
    long long nforce = 0;
    int ngroups = 0;
    for (int s = 0; s < n_sys; ++s) {
        DSys &S = c->ds[s];
        S.grp0 = S.ngrp = 0;
        if (c->pair) {
            // the system's replicas are consecutive, and so are their list force CTAs
            S.fcta0 = c->dr[S.rep0].fcta0;
            S.fcta1 = c->dr[S.rep0 + c->hs[s].P - 1].fcta0 + (c->hs[s].N + list_atoms(lanes) - 1) / list_atoms(lanes);
            nforce = S.fcta1;
            S.grp0 = ngroups;
            S.ngrp = (S.fcta1 - S.fcta0 + kRedGroup - 1) / kRedGroup;
            ngroups += S.ngrp;
        } else {
            S.fcta0 = s * ext_gx;
            S.fcta1 = (s + 1) * ext_gx;
            nforce = S.fcta1;
        }
    }

    Dev &d = c->d;
    d.nsys = n_sys;
    d.nrep = nrep;
    d.ncells = ncells;
    d.cap = cap;
    d.stage_cap = stage_cap;
    d.nunits = nlcta;
    d.maxnb = maxnb;
    d.G = G;
    d.Dtot = D;
    d.obs_stride = p->obs_stride;
    d.rebuild_all = p->rebuild_scope;
    d.max_records = p->max_records;
    d.dt = p->dt;
    d.seed = p->seed;
    for (int a = 0; a < nt; ++a) d.mass_mvv[a] = p->mass[a] * kMvv2e;

    MdLaunch &m = c->ml;
    m.mixed = c->mixed;
    m.pair = c->pair;
    m.n_icta = icta;
    m.n_ccta = ccta;
    m.n_ecta = ext_gx;
    m.nP = 0;
    for (int s = 0; s < n_sys; ++s) {
        bool seen = false;
        for (int u = 0; u < m.nP; ++u) seen |= (m.Pvals[u] == c->hs[s].P);
        if (!seen) {
            if (m.nP == 8) return bail(fail(QTB_ERR_ARG, "at most 8 distinct bead counts per context"));
            m.Pvals[m.nP++] = c->hs[s].P;
        }
    }
    m.nm_big = nm_big;
    // one-bead pair systems fuse the next step's first half into the step kernel
    // (with cells, behind a grid barrier after the cells' updates)
    m.fused = c->pair ? 1 : 0;
    for (int s = 0; s < n_sys; ++s)
        if (c->hs[s].P != 1) m.fused = 0;
    if (integrate_prepare(m) != cudaSuccess)
        return bail(fail(QTB_ERR_CUDA, "cannot reserve shared memory for the ring-polymer integrator"));

    // tables
    std::vector<double> rot;
    for (int s = 0; s < n_sys; ++s) {
        const DSys &S = c->ds[s];
        for (int k = 0; k < S.P; ++k) {
            const double w = 2.0 * S.wP * std::sin(kPi * k / S.P);
            const double ph = 0.5 * p->dt * w;
            if (w == 0.0) {
                rot.push_back(1.0);
                rot.push_back(0.5 * p->dt);
                rot.push_back(0.0);
            } else {
                rot.push_back(std::cos(ph));
                rot.push_back(std::sin(ph) / w);
                rot.push_back(-w * std::sin(ph));
            }
        }
    }
    std::vector<double> hdt(nt), osig((size_t)n_sys * kMaxTypes, 0.0);
    for (int a = 0; a < nt; ++a) hdt[a] = 0.5 * p->dt / (p->mass[a] * kMvv2e);
    for (int s = 0; s < n_sys; ++s)
        for (int a = 0; a < nt; ++a) {
            const double c1 = c->ds[s].c1;
            osig[(size_t)s * kMaxTypes + a] = std::sqrt((1.0 - c1 * c1) / (p->mass[a] * kMvv2e));
        }
    auto as_real = [&](const std::vector<double> &v) -> void * {
        if (c->mixed) {
            std::vector<float> f(v.begin(), v.end());
            return upload(c, f);
        }
        return upload(c, v);
    };
    d.rot = as_real(rot);
    d.nmC = as_real(nmC_host);
    d.hdt_m = as_real(hdt);
    d.osig = as_real(osig);
    std::vector<int> typ((size_t)G);
    for (int s = 0; s < n_sys; ++s)
        for (int b = 0; b < c->hs[s].P; ++b)
            for (int i = 0; i < c->hs[s].N; ++i) typ[(size_t)c->ds[s].g0 + (size_t)b * c->hs[s].N + i] = sys[s].type[i];
    d.typ = upload(c, typ);
    d.rep = upload(c, c->dr);
    d.cell_rep = upload(c, c->cell_rep);
    d.lcta_rep = upload(c, c->lcta_rep);
    d.icta_sys = upload(c, c->icta_sys);
    d.ccta_sys = ccta ? upload(c, c->ccta_sys) : nullptr;
    d.sys = upload(c, c->ds);
    const size_t psz = c->pair && c->mixed ? 4 : c->rsz;
    d.x = c->alloc(psz * 3 * (size_t)G);
    d.v = c->alloc(c->rsz * 3 * (size_t)G);
    d.f = c->alloc(c->rsz * 3 * (size_t)G);
    d.cnt = (int *)c->alloc(sizeof(int) * std::max(ncells, 1));
    d.ccount = (int *)c->alloc(sizeof(int) * std::max(ncells, 1));
    d.cidx = (int *)c->alloc(sizeof(int) * (size_t)std::max(ncells, 1) * cap);
    d.cpos = c->alloc((c->mixed ? 16 : 32) * (size_t)std::max(ncells, 1) * cap);
    if (c->pair) {
        for (int k = 0; k < 2; ++k) d.pos[k] = c->alloc((c->mixed ? 16 : 32) * (size_t)G);
        d.xref = c->alloc(psz * 3 * (size_t)G);
        d.nbr = (unsigned *)c->alloc(sizeof(unsigned) * (size_t)G * maxnb);
        d.nnb = (int *)c->alloc(sizeof(int) * (size_t)G);
        if (!d.pos[0] || !d.pos[1] || !d.xref || !d.nbr || !d.nnb)
            return bail(fail(QTB_ERR_OOM, "neighbour-list allocation failed"));
        // the type word of both packed position buffers (positions follow)
        for (int k = 0; k < 2; ++k) {
            if (c->mixed) {
                std::vector<int4> pk((size_t)G);
                for (size_t g = 0; g < (size_t)G; ++g) pk[g] = make_int4(0, 0, 0, typ[g]);
                cudaMemcpyAsync(d.pos[k], pk.data(), sizeof(int4) * G, cudaMemcpyHostToDevice, c->st);
            } else {
                std::vector<double> pk(4 * (size_t)G, 0.0);
                for (size_t g = 0; g < (size_t)G; ++g) pk[4 * g + 3] = (double)typ[g];
                cudaMemcpyAsync(d.pos[k], pk.data(), sizeof(double) * 4 * G, cudaMemcpyHostToDevice, c->st);
            }
            if (cudaStreamSynchronize(c->st) != cudaSuccess) return bail(fail(QTB_ERR_CUDA, "upload failed"));
        }
        cudaMemsetAsync(d.nnb, 0, sizeof(int) * (size_t)G, c->st);
    }
    d.flag = (unsigned *)c->alloc(2 * sizeof(unsigned));
    d.rflag = (unsigned *)c->alloc(2 * sizeof(unsigned) * n_sys);
    if (!d.rflag) return bail(fail(QTB_ERR_OOM, "device allocation failed"));
    cudaMemsetAsync(d.rflag, 0, 2 * sizeof(unsigned) * n_sys, c->st);
    d.gbar = (unsigned *)c->alloc(2 * sizeof(unsigned));
    d.nrebuild = (unsigned long long *)c->alloc(sizeof(unsigned long long));
    if (!d.flag || !d.gbar || !d.nrebuild) return bail(fail(QTB_ERR_OOM, "device allocation failed"));
    cudaMemsetAsync(d.nrebuild, 0, sizeof(unsigned long long), c->st);
    cudaMemsetAsync(d.flag, 0, 2 * sizeof(unsigned), c->st);
    cudaMemsetAsync(d.gbar, 0, 2 * sizeof(unsigned), c->st);
    d.eta = c->alloc(c->rsz * (size_t)kBlockSteps * (size_t)D);
    d.eta_blocks = 1;
    d.part = (double *)c->alloc(sizeof(double) * kNQ * (size_t)std::max(nforce, 1LL));
    d.gpart = (double *)c->alloc(sizeof(double) * kNQ * (size_t)std::max(ngroups, 1));
    d.gdone = (unsigned *)c->alloc(sizeof(unsigned) * (size_t)std::max(ngroups, 1));
    if (!d.gpart || !d.gdone) return bail(fail(QTB_ERR_OOM, "device allocation failed"));
    cudaMemsetAsync(d.gdone, 0, sizeof(unsigned) * (size_t)std::max(ngroups, 1), c->st);
    d.ipart = (double *)c->alloc(sizeof(double) * kNQ * (size_t)icta);
    d.latest = (double *)c->alloc(sizeof(double) * QTB_NREC * n_sys);
    d.series = (double *)c->alloc(sizeof(double) * QTB_NREC * (size_t)n_sys * p->max_records);
    d.clock = (long long *)c->alloc(sizeof(long long));
    d.err = (unsigned *)c->alloc(sizeof(unsigned));
    d.done = (unsigned *)c->alloc(sizeof(unsigned) * n_sys);
    if (!d.done) return bail(fail(QTB_ERR_OOM, "device allocation failed"));
    cudaMemsetAsync(d.done, 0, sizeof(unsigned) * n_sys, c->st);
    d.npt = nullptr;
    if (p->npt) {
        std::vector<DNpt> cells((size_t)n_sys);
        for (int s = 0; s < n_sys; ++s) {
            DNpt &C = cells[s];
            memset(&C, 0, sizeof C);
            C.lam = C.lam_rb = 1.0;
            C.W = p->cell_mass;
            C.pext = p->pressure;
            C.ce = std::exp(-p->cell_gamma * p->dt);
            C.sige = std::sqrt((1.0 - C.ce * C.ce) * C.W * kBoltz * sys[s].T);
            C.alpha = 1.0 + 1.0 / sys[s].n_atoms;  // 1 + 3/N_f, N_f = 3N
            C.V0 = sys[s].box[0] * sys[s].box[1] * sys[s].box[2];
            C.e1 = C.g1 = C.e2 = C.g2 = 1.0;
            C.a1 = C.a2 = 0.5 * p->dt;
            C.e1f = C.g1f = C.e2f = C.g2f = C.lamf = 1.0f;
            C.a1f = C.a2f = (float)(0.5 * p->dt);
            C.inv_wf = (float)(1.0 / p->cell_mass);
            C.rb_tol = kNptCellSkin * c->skins[s] / (p->r_cut + c->skins[s]);
            C.lam_old = C.inv_lam = 1.0;
            C.lam_oldf = C.inv_lamf = 1.0f;
            C.on = 1;
        }
        d.npt = upload(c, cells);
        if (!d.npt) return bail(fail(QTB_ERR_OOM, "device allocation failed"));
    }
    if (ccta) {
        d.cpart = (double *)c->alloc(sizeof(double) * 6 * (size_t)ccta);  // kCenQ per CTA
        d.cdone = (unsigned *)c->alloc(sizeof(unsigned) * n_sys);
        if (!d.cpart || !d.cdone || !d.ccta_sys) return bail(fail(QTB_ERR_OOM, "device allocation failed"));
        cudaMemsetAsync(d.cdone, 0, sizeof(unsigned) * n_sys, c->st);
    }
    c->dspec = (DSpec *)c->alloc(sizeof(DSpec) * n_sys);
    if (!d.x || !d.v || !d.f || !d.cnt || !d.ccount || !d.cidx || !d.cpos || !d.eta || !d.part || !d.ipart ||
        !d.latest || !d.series || !d.clock || !d.err || !d.typ || !d.sys || !c->dspec)
        return bail(fail(QTB_ERR_OOM, "device allocation failed"));
    cudaMemsetAsync(d.cnt, 0, sizeof(int) * std::max(ncells, 1), c->st);
    cudaMemsetAsync(d.ccount, 0, sizeof(int) * std::max(ncells, 1), c->st);
    cudaMemsetAsync(d.clock, 0, sizeof(long long), c->st);
    cudaMemsetAsync(d.err, 0, sizeof(unsigned), c->st);
    cudaMemsetAsync(d.series, 0, sizeof(double) * QTB_NREC * (size_t)n_sys * p->max_records, c->st);
    cudaMemsetAsync(d.v, 0, c->rsz * 3 * (size_t)G, c->st);
    cudaMemsetAsync(d.eta, 0, c->rsz * (size_t)kBlockSteps * (size_t)D, c->st);
    c->dclock = 0;
    for (int s = 0; s < n_sys; ++s) {
        rc = upload_state(c, s, sys[s].pos, sys[s].vel);
        if (rc) return bail(rc);
    }
    rc = rebuild_filters(c);
    if (rc) return bail(rc);
    rc = refresh_forces(c);
    if (rc) return bail(rc);
    rc = check_err_word(c);
    if (rc) return bail(rc);
    *out = c;
    return QTB_OK;
}

void qtb_destroy(qtb_ctx *c) { delete c; }

int qtb_set_filter(qtb_ctx *c, int sys, int mode, int n_taps, double omega_max)
{
    if (!c) return fail(QTB_ERR_ARG, "null context");
    if (mode < 0 || mode > 3) return fail(QTB_ERR_ARG, "unknown noise mode %d", mode);
    if (mode == QTB_NOISE_QTB_PIMD_MLP && !c->kmodel) return fail(QTB_ERR_STATE, "no learned kappa_P model is set");
    if (mode != QTB_NOISE_WHITE && (n_taps < 1 || n_taps % 2 == 0))
        return fail(QTB_ERR_ARG, "n_taps must be odd and >= 1");
    const int ns = (int)c->hs.size();
    if (sys < -1 || sys >= ns) return fail(QTB_ERR_ARG, "system %d out of range", sys);
    for (int s = (sys < 0 ? 0 : sys); s < (sys < 0 ? ns : sys + 1); ++s) {
        if (mode == QTB_NOISE_QTB && c->hs[s].P != 1)
            return fail(QTB_ERR_ARG, "system %d: QTB needs n_beads = 1 (use QTB_PIMD)", s);
    }
    for (int s = (sys < 0 ? 0 : sys); s < (sys < 0 ? ns : sys + 1); ++s) {
        c->hs[s].mode = mode;
        c->hs[s].n_taps = (mode == QTB_NOISE_WHITE) ? 1 : n_taps;
        c->hs[s].omega_max = omega_max;
    }
    return rebuild_filters(c);
}

// one force evaluation (lists rebuilt where needed, record of the current step)
// for all the states set since the last one
static int ensure_fresh(qtb_ctx *c)
{
    if (!c->stale) return QTB_OK;
    c->stale = false;
    return refresh_forces(c);
}

int qtb_step_n(qtb_ctx *c, long long n)
{
    if (!c) return fail(QTB_ERR_ARG, "null context");
    if (n < 0) return fail(QTB_ERR_ARG, "n_steps < 0");
    if (int rc = ensure_fresh(c)) return rc;
    while (n > 0) {
        const long long b = floor_div(c->step, kBlockSteps);
        const int j = (int)(c->step - b * kBlockSteps);
        if (j == 0 && n >= kBlockSteps) {
            // the graph generates white block b + Kb and filters block b (filter), or
            // generates a new segment when b starts one (Fourier segments)
            if (c->gen == QTB_GEN_FOURIER) {
                if (b % c->seg_blocks != 0) ensure_eta(c, b);  // the segment b lies in
            } else {
                ensure_ring(c, b - c->d.Kb, b + c->d.Kb - 1);
            }
            set_clock(c, b);
            if (c->graph_dirty || !c->gexec) {
                int rc = build_graph(c);
                if (rc) return rc;
            }
            CUDA_TRY(cudaGraphLaunch(c->gexec, c->st));
            c->prof_launched = c->profiling;
            c->ring_hi = b + c->d.Kb;
            c->ring_lo = c->ring_hi - c->d.nslots + 1;
            c->eta_blk = b;
            c->eta_seg = floor_div(b, c->seg_blocks);
            c->dclock = b + 1;
            c->step += kBlockSteps;
            n -= kBlockSteps;
            continue;
        }
        ensure_eta(c, b);
        const long long mcount = std::min<long long>(n, kBlockSteps - j);
        int rc = run_steps(c, j, (int)mcount, false);
        if (rc) return rc;
        c->step += mcount;
        n -= mcount;
        if (j + mcount == kBlockSteps) {
            launch_tick(c->d, c->st);
            c->dclock = b + 1;
        }
        CUDA_TRY(cudaGetLastError());
    }
    CUDA_TRY(cudaGetLastError());
    return QTB_OK;
}

int qtb_set_generator(qtb_ctx *c, int generator, int segment_blocks)
{
    if (!c) return fail(QTB_ERR_ARG, "null context");
    if (generator != QTB_GEN_FILTER && generator != QTB_GEN_FOURIER) return fail(QTB_ERR_ARG, "unknown generator");
    const int M = generator == QTB_GEN_FOURIER ? segment_blocks : 1;
    if (M != 1 && M != 2 && M != 4 && M != 8) return fail(QTB_ERR_ARG, "segment_blocks must be 1, 2, 4 or 8");
    CUDA_TRY(cudaStreamSynchronize(c->st));
    if (M != c->seg_blocks) {
        void *eta = c->alloc(c->rsz * (size_t)kBlockSteps * M * (size_t)c->d.Dtot);
        if (!eta) return fail(QTB_ERR_OOM, "noise segment allocation failed");
        CUDA_TRY(cudaMemsetAsync(eta, 0, c->rsz * (size_t)kBlockSteps * M * (size_t)c->d.Dtot, c->st));
        c->release(c->d.eta);
        c->d.eta = eta;
    }
    const int old_gen = c->gen, old_m = c->seg_blocks;
    c->gen = generator;
    c->seg_blocks = M;
    c->d.eta_blocks = M;
    int rc = rebuild_filters(c);
    if (rc) {
        c->gen = old_gen;
        c->seg_blocks = c->d.eta_blocks = old_m;
        if (old_m != M) {
            c->release(c->d.eta);
            c->d.eta = c->alloc(c->rsz * (size_t)kBlockSteps * old_m * (size_t)c->d.Dtot);
        }
        rebuild_filters(c);
        return rc;
    }
    return QTB_OK;
}

int qtb_sync(qtb_ctx *c)
{
    if (!c) return fail(QTB_ERR_ARG, "null context");
    if (int rc0 = ensure_fresh(c)) return rc0;
    return check_err_word(c);
}

int qtb_observables(qtb_ctx *c, int sys, double *out)
{
    if (!c || !out) return fail(QTB_ERR_ARG, "null argument");
    if (sys < 0 || sys >= (int)c->hs.size()) return fail(QTB_ERR_ARG, "system %d out of range", sys);
    if (int rc0 = ensure_fresh(c)) return rc0;
    // the error word and the record in one synchronisation (on an error the
    // record is returned as it is, with the error code)
    unsigned e = 0;
    CUDA_TRY(cudaMemcpyAsync(&e, c->d.err, sizeof e, cudaMemcpyDeviceToHost, c->st));
    CUDA_TRY(cudaMemcpyAsync(out, c->d.latest + (size_t)sys * QTB_NREC, sizeof(double) * QTB_NREC,
                             cudaMemcpyDeviceToHost, c->st));
    CUDA_TRY(cudaStreamSynchronize(c->st));
    return decode_err_word(c, e);
}

int qtb_get_series(qtb_ctx *c, int sys, double *out, int max, int *n_out)
{
    if (!c || !out || !n_out) return fail(QTB_ERR_ARG, "null argument");
    if (sys < 0 || sys >= (int)c->hs.size()) return fail(QTB_ERR_ARG, "system %d out of range", sys);
    if (int rc0 = ensure_fresh(c)) return rc0;
    int rc = check_err_word(c);
    if (rc) return rc;
    const long long total = c->step / c->p.obs_stride;
    long long n = std::min<long long>(total, std::min(c->p.max_records, max));
    const int ns = (int)c->hs.size();
    std::vector<double> all((size_t)c->p.max_records * ns * QTB_NREC);
    CUDA_TRY(cudaMemcpyAsync(all.data(), c->d.series, sizeof(double) * all.size(), cudaMemcpyDeviceToHost, c->st));
    CUDA_TRY(cudaStreamSynchronize(c->st));
    for (long long i = 0; i < n; ++i) {
        const long long r = total - n + i;
        const int slot = (int)(r % c->p.max_records);
        memcpy(out + i * QTB_NREC, all.data() + ((size_t)slot * ns + sys) * QTB_NREC, sizeof(double) * QTB_NREC);
    }
    *n_out = (int)n;
    return QTB_OK;
}

int qtb_get_state(qtb_ctx *c, int sys, double *pos, double *vel)
{
    if (!c) return fail(QTB_ERR_ARG, "null context");
    if (sys < 0 || sys >= (int)c->hs.size()) return fail(QTB_ERR_ARG, "system %d out of range", sys);
    if (int rc0 = ensure_fresh(c)) return rc0;
    int rc = check_err_word(c);
    if (rc) return rc;
    if (pos && (rc = download(c, sys, 0, pos))) return rc;
    if (vel && (rc = download(c, sys, 1, vel))) return rc;
    return QTB_OK;
}

int qtb_set_state(qtb_ctx *c, int sys, const double *pos, const double *vel)
{
    if (!c) return fail(QTB_ERR_ARG, "null context");
    if (sys < 0 || sys >= (int)c->hs.size()) return fail(QTB_ERR_ARG, "system %d out of range", sys);
    int rc = upload_state(c, sys, pos, vel);
    if (rc) return rc;
    c->stale = true;  // forces and the record follow at the next call that needs them
    return QTB_OK;
}

int qtb_get_forces(qtb_ctx *c, int sys, double *f)
{
    if (!c || !f) return fail(QTB_ERR_ARG, "null argument");
    if (sys < 0 || sys >= (int)c->hs.size()) return fail(QTB_ERR_ARG, "system %d out of range", sys);
    if (int rc0 = ensure_fresh(c)) return rc0;
    int rc = check_err_word(c);
    if (rc) return rc;
    return download(c, sys, 2, f);
}

int qtb_get_taps(qtb_ctx *c, int sys, double *h, int max, int *n_out)
{
    if (!c || !h || !n_out) return fail(QTB_ERR_ARG, "null argument");
    if (sys < 0 || sys >= (int)c->hs.size()) return fail(QTB_ERR_ARG, "system %d out of range", sys);
    const DSys &S = c->ds[sys];
    const int n = std::min(max, S.K + 1);
    CUDA_TRY(cudaMemcpyAsync(h, c->d_taps64 + S.taps0, sizeof(double) * n, cudaMemcpyDeviceToHost, c->st));
    CUDA_TRY(cudaStreamSynchronize(c->st));
    *n_out = n;
    return QTB_OK;
}

int qtb_get_noise(qtb_ctx *c, int sys, double *out, long long *block_out)
{
    if (!c || !out) return fail(QTB_ERR_ARG, "null argument");
    if (sys < 0 || sys >= (int)c->hs.size()) return fail(QTB_ERR_ARG, "system %d out of range", sys);
    const long long b = floor_div(c->step, kBlockSteps);
    ensure_eta(c, b);
    CUDA_TRY(cudaGetLastError());
    const DSys &S = c->ds[sys];
    const int D = 3 * S.N * S.P;
    // rows of block b in the noise buffer (Fourier segments hold seg_blocks blocks)
    const size_t r0 = (size_t)(b - floor_div(b, c->seg_blocks) * c->seg_blocks) * kBlockSteps;
    if (c->mixed) {
        std::vector<float> buf((size_t)kBlockSteps * D);
        for (int j = 0; j < kBlockSteps; ++j)
            CUDA_TRY(cudaMemcpyAsync(buf.data() + (size_t)j * D, (const float *)c->d.eta + (r0 + j) * c->d.Dtot + S.dof0,
                                     sizeof(float) * D, cudaMemcpyDeviceToHost, c->st));
        CUDA_TRY(cudaStreamSynchronize(c->st));
        for (size_t t = 0; t < buf.size(); ++t) out[t] = buf[t];
    } else {
        for (int j = 0; j < kBlockSteps; ++j)
            CUDA_TRY(cudaMemcpyAsync(out + (size_t)j * D, (const double *)c->d.eta + (r0 + j) * c->d.Dtot + S.dof0,
                                     sizeof(double) * D, cudaMemcpyDeviceToHost, c->st));
        CUDA_TRY(cudaStreamSynchronize(c->st));
    }
    if (block_out) *block_out = b;
    return check_err_word(c);
}

int qtb_set_profiling(qtb_ctx *c, int enable)
{
    if (!c) return fail(QTB_ERR_ARG, "null context");
    c->profiling = (enable != 0);
    c->prof_launched = false;
    c->graph_dirty = true;
    return QTB_OK;
}

int qtb_kernel_times(qtb_ctx *c, double *mean_ms, int *counts, int n_classes)
{
    if (!c || !mean_ms || !counts || n_classes < 1) return fail(QTB_ERR_ARG, "null argument");
    if (!c->prof_launched) return fail(QTB_ERR_STATE, "no profiled 256-step block has run");
    CUDA_TRY(cudaStreamSynchronize(c->st));
    for (int k = 0; k < n_classes; ++k) {
        mean_ms[k] = 0.0;
        counts[k] = 0;
    }
    for (size_t pr = 0; pr < c->ev_pairs; ++pr) {
        const int k = c->ev_cls[pr];
        if (k >= n_classes) continue;
        float ms = 0.f;
        CUDA_TRY(cudaEventElapsedTime(&ms, c->ev[2 * pr], c->ev[2 * pr + 1]));
        mean_ms[k] += ms;
        counts[k] += 1;
    }
    for (int k = 0; k < n_classes; ++k)
        if (counts[k]) mean_ms[k] /= counts[k];
    return QTB_OK;
}

int qtb_set_kappa_model(qtb_ctx *c, const qtb_kappa_model *model)
{
    if (!c) return fail(QTB_ERR_ARG, "null context");
    c->kmodel = model;
    return QTB_OK;
}

int qtb_filter_source(qtb_ctx *c, int sys, int *source)
{
    if (!c || !source) return fail(QTB_ERR_ARG, "null argument");
    if (sys < 0 || sys >= (int)c->hs.size()) return fail(QTB_ERR_ARG, "system %d out of range", sys);
    *source = c->ksrc[sys];
    return QTB_OK;
}

int qtb_rebuild_lists(qtb_ctx *c)
{
    if (!c) return fail(QTB_ERR_ARG, "null context");
    if (!c->pair) return QTB_OK;
    // the next call that needs the forces rebuilds every system's lists, the
    // way the first evaluation after qtb_init does
    c->lists_built = false;
    c->stale = true;
    return QTB_OK;
}

int qtb_list_rebuilds(qtb_ctx *c, long long *count)
{
    if (!c || !count) return fail(QTB_ERR_ARG, "null argument");
    if (int rc0 = ensure_fresh(c)) return rc0;
    unsigned long long n = 0;
    if (c->pair) {
        CUDA_TRY(cudaMemcpyAsync(&n, c->d.nrebuild, sizeof n, cudaMemcpyDeviceToHost, c->st));
        CUDA_TRY(cudaStreamSynchronize(c->st));
    }
    *count = (long long)n;
    return QTB_OK;
}

int qtb_wait_selftest(qtb_ctx *c, int *gave_up, double *ms)
{
    if (!c || !gave_up || !ms) return fail(QTB_ERR_ARG, "null argument");
    if (int rc = check_err_word(c)) return rc;
    if (!c->d_selftest) {
        c->d_selftest = (unsigned *)c->alloc(2 * sizeof(unsigned));
        if (!c->d_selftest) return fail(QTB_ERR_OOM, "device allocation failed");
    }
    CUDA_TRY(cudaMemsetAsync(c->d_selftest, 0, 2 * sizeof(unsigned), c->st));
    cudaEvent_t a, b;
    CUDA_TRY(cudaEventCreate(&a));
    CUDA_TRY(cudaEventCreate(&b));
    cudaEventRecord(a, c->st);
    launch_wait_selftest(c->d_selftest, c->st);
    cudaEventRecord(b, c->st);
    unsigned h[2] = {0u, 0u};
    cudaError_t e = cudaMemcpyAsync(h, c->d_selftest, sizeof h, cudaMemcpyDeviceToHost, c->st);
    if (e == cudaSuccess) e = cudaStreamSynchronize(c->st);
    float t = 0.f;
    if (e == cudaSuccess) e = cudaEventElapsedTime(&t, a, b);
    cudaEventDestroy(a);
    cudaEventDestroy(b);
    if (e != cudaSuccess) return fail(QTB_ERR_CUDA, "wait self-test: %s", cudaGetErrorString(e));
    *gave_up = h[1] != 0u;
    *ms = t;
    return QTB_OK;
}

int qtb_get_step(qtb_ctx *c, long long *step)
{
    if (!c || !step) return fail(QTB_ERR_ARG, "null argument");
    *step = c->step;
    return QTB_OK;
}

int qtb_get_cell(qtb_ctx *c, int sys, double *box, double *p_e)
{
    if (!c) return fail(QTB_ERR_ARG, "null context");
    if (sys < 0 || sys >= (int)c->hs.size()) return fail(QTB_ERR_ARG, "system %d out of range", sys);
    if (int rc0 = ensure_fresh(c)) return rc0;
    int rc = check_err_word(c);
    if (rc) return rc;
    double lam = 1.0, pe = 0.0;
    if (c->d.npt) {
        DNpt C;
        CUDA_TRY(cudaMemcpyAsync(&C, c->d.npt + sys, sizeof C, cudaMemcpyDeviceToHost, c->st));
        CUDA_TRY(cudaStreamSynchronize(c->st));
        lam = C.lam;
        pe = C.peps;
    }
    if (box)
        for (int k = 0; k < 3; ++k) box[k] = c->hs[sys].box[k] * lam;
    if (p_e) *p_e = pe;
    return QTB_OK;
}

int qtb_set_cell(qtb_ctx *c, int sys, const double *box, double p_e)
{
    if (!c || !box) return fail(QTB_ERR_ARG, "null argument");
    if (sys < 0 || sys >= (int)c->hs.size()) return fail(QTB_ERR_ARG, "system %d out of range", sys);
    if (!c->d.npt) return fail(QTB_ERR_ARG, "qtb_set_cell: not an isothermal-isobaric context");
    const double *ref = c->hs[sys].box;
    const double lam = box[0] / ref[0];
    for (int k = 0; k < 3; ++k)
        if (!(std::fabs(box[k] / ref[k] - lam) <= 1e-12 * lam))
            return fail(QTB_ERR_ARG, "qtb_set_cell: the cell is isotropic (edges proportional to the initial ones)");
    if (!std::isfinite(lam) || !(lam >= kCellMinScale) || !std::isfinite(p_e))
        return fail(QTB_ERR_ARG, "qtb_set_cell: edges below %.2f of the initial ones or not finite", kCellMinScale);
    if (int rc0 = ensure_fresh(c)) return rc0;
    if (int rc = check_err_word(c)) return rc;
    DNpt C;
    CUDA_TRY(cudaMemcpyAsync(&C, c->d.npt + sys, sizeof C, cudaMemcpyDeviceToHost, c->st));
    CUDA_TRY(cudaStreamSynchronize(c->st));
    C.lam = lam;
    C.lamf = (float)lam;
    C.peps = p_e;  // whether the closing half kick is due stays as it is
    CUDA_TRY(cudaMemcpyAsync(c->d.npt + sys, &C, sizeof C, cudaMemcpyHostToDevice, c->st));
    CUDA_TRY(cudaStreamSynchronize(c->st));
    // positions are stored relative to the cell and scale with it; every list is
    // rebuilt and the forces and record evaluated again at the next call that
    // needs them
    if (c->pair) c->lists_built = false;
    c->stale = true;
    return QTB_OK;
}

int qtb_fp32_peak(double *tflops, double *ms)
{
    if (!tflops) return fail(QTB_ERR_ARG, "qtb_fp32_peak: null tflops");
    const int rc = measure_fp32_peak(tflops, ms);
    if (rc == QTB_ERR_OOM) return fail(rc, "qtb_fp32_peak: device allocation failed");
    if (rc != QTB_OK) return fail(rc, "qtb_fp32_peak: CUDA error %s", cudaGetErrorString(cudaGetLastError()));
    return QTB_OK;
}

int qtb_kappa_solve(int P, int n, double y_max, double y0, double *F)
{
    if (P < 1 || n < 8 || !(y_max > 0) || !(y0 > 0) || !F) return fail(QTB_ERR_ARG, "qtb_kappa_solve: bad arguments");
    if (P == 1) {
        const double dts = std::asinh(y_max / y0) / (n - 1);
        for (int i = 0; i < n; ++i) {
            const double x = y0 * std::sinh(i * dts);
            F[i] = (x < 1e-6) ? 1.0 + x * x / 12.0 : x * (0.5 + 1.0 / std::expm1(x));
        }
        return QTB_OK;
    }
    const int rows = 2 * n - 1;
    double *A = nullptr, *b = nullptr, *M = nullptr, *r = nullptr;
    unsigned *err = nullptr;
    size_t need = sizeof(double) * ((size_t)rows * n + rows + (size_t)n * n + n + rows + n) + 16;
    char *base = nullptr;
    CUDA_TRY(cudaMalloc(&base, need));
    A = (double *)base;
    b = A + (size_t)rows * n;
    M = b + rows;
    r = M + (size_t)n * n;
    double *work = r + n;
    err = (unsigned *)(work + rows + n);
    cudaMemset(err, 0, sizeof(unsigned));
    launch_kappa_solve(P, n, y_max, y0, A, b, M, r, work, err, 0);
    unsigned e = 0;
    cudaError_t ce = cudaGetLastError();
    if (ce == cudaSuccess) ce = cudaMemcpy(F, r, sizeof(double) * n, cudaMemcpyDeviceToHost);
    if (ce == cudaSuccess) ce = cudaMemcpy(&e, err, sizeof e, cudaMemcpyDeviceToHost);
    cudaFree(base);
    if (ce != cudaSuccess) return fail(QTB_ERR_CUDA, "qtb_kappa_solve: %s", cudaGetErrorString(ce));
    if (e) return fail(QTB_ERR_SOLVE, "qtb_kappa_solve: non-positive pivot");
    return QTB_OK;
}

}  // extern "C"
