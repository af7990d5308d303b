// autotune.cu -- qtb_autotune: launch shapes and neighbour-list batching chosen
// by timing whole 256-step blocks of the caller's systems on the device.
#include <cuda_runtime.h>

#include <cmath>
#include <string>
#include <vector>

#include "../../include/qtb.h"
#include "qtb_dev.cuh"
#include "qtb_kernels.cuh"

namespace {

// mean device time of one MD step (ms) for parameters q, or a negative value
double time_config(const qtb_system *sys, int n_sys, const qtb_params *q, void *stream, int mode, int n_taps,
                   double wmax, int n_blocks, int *rc_out)
{
    qtb_ctx *c = nullptr;
    int rc = qtb_init(&c, sys, n_sys, q, stream);
    if (rc == QTB_OK && mode != QTB_NOISE_WHITE) rc = qtb_set_filter(c, -1, mode, n_taps, wmax);
    // warm-up as long as the timed run: graph capture, and the rebuild rate of a
    // system that has left its initial configuration
    if (rc == QTB_OK) rc = qtb_step_n(c, (long long)n_blocks * qtb::kBlockSteps);
    if (rc == QTB_OK) rc = qtb_sync(c);
    double ms = -1.0;
    if (rc == QTB_OK) {
        cudaStream_t st = (cudaStream_t)stream;
        cudaEvent_t a, b;
        cudaEventCreate(&a);
        cudaEventCreate(&b);
        // the context's own stream when the caller gave none: time on the device clock of
        // the whole run instead (synchronising brackets)
        cudaDeviceSynchronize();
        cudaEventRecord(a, st);
        rc = qtb_step_n(c, (long long)n_blocks * qtb::kBlockSteps);
        if (rc == QTB_OK) rc = qtb_sync(c);
        cudaDeviceSynchronize();
        cudaEventRecord(b, st);
        cudaEventSynchronize(b);
        float t = 0.f;
        if (rc == QTB_OK && cudaEventElapsedTime(&t, a, b) == cudaSuccess) ms = t / (n_blocks * qtb::kBlockSteps);
        cudaEventDestroy(a);
        cudaEventDestroy(b);
    }
    if (c) qtb_destroy(c);
    *rc_out = rc;
    return ms;
}

}  // namespace

extern "C" int qtb_autotune(const qtb_system *sys_in, int n_sys, const qtb_params *p, void *stream, int noise_mode,
                            int n_taps, double omega_max, int n_blocks, int equil_blocks, qtb_params *best,
                            qtb_tuning *result)
{
    if (!sys_in || n_sys < 1 || !p || !best || !result || n_blocks < 1 || equil_blocks < 0)
        return qtb::set_last_error(QTB_ERR_ARG, "qtb_autotune: bad arguments");
    if (p->potential != QTB_POT_PAIR) return qtb::set_last_error(QTB_ERR_ARG, "qtb_autotune: pair potential only");
    // Steady state: equilibrate once with the default parameters; every candidate
    // then starts from that thermalised configuration, its lists built on it, so
    // that the timing sees the list lengths and the rebuild rate of a long run
    // rather than those of the initial lattice.
    std::vector<qtb_system> sys(sys_in, sys_in + n_sys);
    std::vector<std::vector<double>> xs(n_sys), vs(n_sys);
    if (equil_blocks > 0) {
        qtb_params q0 = *p;
        q0.skin = 0.0;
        q0.nm_layout = 0;
        q0.list_lanes = 0;
        q0.rebuild_scope = 0;
        qtb_ctx *c = nullptr;
        int rc = qtb_init(&c, sys_in, n_sys, &q0, stream);
        if (rc == QTB_OK && noise_mode != QTB_NOISE_WHITE) rc = qtb_set_filter(c, -1, noise_mode, n_taps, omega_max);
        if (rc == QTB_OK) rc = qtb_step_n(c, (long long)equil_blocks * qtb::kBlockSteps);
        for (int s = 0; s < n_sys && rc == QTB_OK; ++s) {
            const size_t n3 = 3 * (size_t)sys_in[s].n_atoms * sys_in[s].n_beads;
            xs[s].resize(n3);
            vs[s].resize(n3);
            rc = qtb_get_state(c, s, xs[s].data(), vs[s].data());
            sys[s].pos = xs[s].data();
            sys[s].vel = vs[s].data();
        }
        if (c) qtb_destroy(c);
        if (rc != QTB_OK) return rc;
    }
    bool beads = false;
    for (int s = 0; s < n_sys; ++s) beads |= sys_in[s].n_beads > 1;
    const double skins[] = {0.5, 0.8, 1.2, 1.6};
    const int lanes[] = {8, 16, 32};
    const int layouts[] = {1, 2};
    const int n_scope = n_sys > 1 ? 2 : 1;
    double best_ms = -1.0;
    int tried = 0, rc = QTB_OK;
    qtb_params q = *p;
    q.skin = 0.0;
    q.nm_layout = 0;
    q.list_lanes = 0;
    q.rebuild_scope = 0;
    const double def_ms = time_config(sys.data(), n_sys, &q, stream, noise_mode, n_taps, omega_max, n_blocks, &rc);
    if (rc != QTB_OK) return rc;
    *best = q;
    best_ms = def_ms;
    for (double sk : skins) {
        if (!(sk < 0.5 * p->r_cut)) continue;
        for (int ln : lanes)
            for (int li = 0; li < (beads ? 2 : 1); ++li)
                for (int sc = 0; sc < n_scope; ++sc) {
                    q = *p;
                    q.skin = sk;
                    q.list_lanes = ln;
                    q.nm_layout = beads ? layouts[li] : 0;
                    q.rebuild_scope = sc;
                    const double ms = time_config(sys.data(), n_sys, &q, stream, noise_mode, n_taps, omega_max, n_blocks, &rc);
                    ++tried;
                    if (rc != QTB_OK) return rc;
                    if (ms > 0.0 && ms < best_ms) {
                        best_ms = ms;
                        *best = q;
                    }
                }
    }
    result->skin = best->skin;
    result->nm_layout = best->nm_layout;
    result->list_lanes = best->list_lanes;
    result->rebuild_scope = best->rebuild_scope;
    result->ms_per_step = best_ms;
    result->default_ms_per_step = def_ms;
    result->n_tried = tried + 1;
    return QTB_OK;
}
