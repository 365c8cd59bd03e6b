// lf_tune.cu -- autotuner of the single-lattice step (lf_tune in include/lf.h).
//
// Every kernel variant computes the same step (the parity tests run each one
// against the oracle); they differ in how the lattice is mapped to the GPU:
// CTA width and rows per segment of the 2D row marches, tile shape and planes
// per segment of the 3D force pass.  The tuner times each candidate on a
// scratch context of the same lattice, stencil, precision and parameters
// (so the caller's state is never touched), keeps the fastest, and caches
// the choice per (device, lattice, stencil, precision, walls, hydrodynamics)
// for the life of the process.
#include <map>
#include <mutex>
#include <tuple>
#include <vector>

#include "lf_ctx.cuh"

namespace {

using Key = std::tuple<int, int, int, int, int, int, int, int, int>;

struct Choice {
    int variant, param;
    float ms;
    int candidates;
};

std::mutex g_mu;
std::map<Key, Choice> g_cache;

Key key_of(const lf_ctx* c)
{
    int dev = 0;
    cudaGetDevice(&dev);
    return Key{dev, c->g.d, c->g.nx, c->g.ny, c->g.nz, c->prec, c->g.stencil, c->g.walls, c->params.hydro};
}

// Candidate (variant, param) pairs of a lattice; the first is the library's
// default choice.
std::vector<std::pair<int, int>> candidates(const lf_ctx* c)
{
    std::vector<std::pair<int, int>> v;
    const lf::Geom& g = c->g;
    const bool iso = g.stencil == LF_STENCIL_ISOTROPIC;
    if (g.d == 2) {
        if (iso) {                                   // the isotropic row marches (two lanes in FP32, one), the tile kernel
            const int heights[] = {0, 4, 8, 12, 16, 24, 32, 48, 64};
            for (int w = 0; w < 2; ++w)
                for (int h : heights) {
                    if (c->prec == LF_FP32 && (h == 0 || 2 * h <= g.ny)) v.push_back({LF_VARIANT_MARCH2, (w << 16) | h});
                    if (h <= g.ny) v.push_back({LF_VARIANT_MARCH, (w << 16) | h});
                }
            v.push_back({LF_VARIANT_TILE, 0});
            return v;
        }
        const int heights[] = {0, 1, 2, 3, 4, 6, 8, 12, 16, 24, 32, 48, 64};
        const int var = c->prec == LF_FP32 ? LF_VARIANT_MARCH2 : LF_VARIANT_MARCH;
        for (int w = 0; w < 2; ++w)                  // 0: 128-thread CTAs (120 columns), 1: 64 threads (56)
            for (int h : heights) {
                if (h > 0 && 2 * h > g.ny && var == LF_VARIANT_MARCH2) continue;
                if (h > 0 && h > g.ny) continue;
                v.push_back({var, (w << 16) | h});
            }
        if (c->prec == LF_FP32)
            for (int w = 0; w < 2; ++w) v.push_back({LF_VARIANT_MARCH, w << 16});
        v.push_back({LF_VARIANT_TILE, 0});
        return v;
    }
    // 3D: the three-pass step with its force-pass shapes and segment heights
    // and the phi pass's segment heights, then the fused plane march
    const int planes[] = {0, 8, 16, 32, 64};
    const int phis[] = {0, 32, 64};
    for (int zc : phis) {
        if (zc > g.nz) continue;
        if (iso) {                                   // sliding-sum force pass: two packed z-lanes, one lane on 28x12 (two or one CTA per SM) or 28x28
            const int sels32[] = {4, 0, 1, 3}, sels64[] = {0};
            const int* sels = c->prec == LF_FP32 ? sels32 : sels64;
            const int nsel = c->prec == LF_FP32 ? 4 : 1;
            const int lanes[] = {0, 48, 64, 96, 128, 192};   // planes per lane of the packed form
            for (int phi_form = 0; phi_form < 2; ++phi_form)  // phi pass: register-staged, cp.async-staged (bit 28)
                for (int i = 0; i < nsel; ++i) {
                    const int base = (phi_form << 28) | (zc << 20) | (sels[i] << 16);
                    if (sels[i] == 4) {
                        for (int h : lanes)
                            if (2 * h <= g.nz + 1 || h == 0) v.push_back({LF_VARIANT_SPLIT3, base | h});
                        continue;
                    }
                    for (int h : planes)
                        if (h <= g.nz) v.push_back({LF_VARIANT_SPLIT3, base | h});
                }
        } else if (c->prec == LF_FP64) {
            for (int h : planes)
                if (h <= g.nz) v.push_back({LF_VARIANT_SPLIT3, (zc << 20) | h});
        } else {
            for (int sel = 0; sel < 3; ++sel)        // packed two-lane 28x12, one lane 60x4, one lane 28x12
                for (int h : planes)
                    if (h <= g.nz) v.push_back({LF_VARIANT_SPLIT3, (zc << 20) | (sel << 16) | h});
        }
    }
    v.push_back({LF_VARIANT_MARCH, 0});
    return v;
}

}  // namespace

extern "C" int lf_tune(lf_ctx* c, int reps, int* variant, int* param, double* ms_per_step)
{
    lf::NvtxRange nvtx_range("lf_tune");
    if (!c || reps < 1 || c->ens_member) return LF_EINVAL;
    const Key key = key_of(c);
    {
        std::lock_guard<std::mutex> lock(g_mu);
        auto it = g_cache.find(key);
        if (it != g_cache.end()) {
            c->g.variant = it->second.variant;
            c->g.tune = it->second.param;
            if (variant) *variant = it->second.variant;
            if (param) *param = it->second.param;
            if (ms_per_step) *ms_per_step = it->second.ms;
            return LF_OK;
        }
    }
    int rc = lf::wait_stream(c->stream);
    if (rc != LF_OK) return rc;
    lf_params p = c->params;
    p.workspace = nullptr;
    p.workspace_bytes = 0;
    p.stream = c->stream;
    lf_ctx* tmp = nullptr;
    if ((rc = lf_create(&c->grid, &c->walls, &p, &tmp)) != LF_OK) return rc;
    if (c->t_solver != tmp->t_solver && (rc = lf_set_t_solver(tmp, c->t_solver)) != LF_OK) {
        lf_destroy(tmp);
        return rc;
    }
    // every candidate starts from the scratch context's initial state, so that
    // none of them times a state the earlier trials drove non-finite
    const size_t fb = (size_t)tmp->Q * tmp->g.plane * tmp->esz, pb = (size_t)tmp->g.plane * tmp->esz;
    unsigned char* save = nullptr;
    if (cudaMalloc((void**)&save, fb + 2 * pb) != cudaSuccess) {
        cudaGetLastError();
        lf_destroy(tmp);
        return LF_ENOMEM;
    }
    const int f0 = tmp->fcur, p0 = tmp->pcur, q0 = tmp->tcur;
    cudaMemcpyAsync(save, tmp->f[f0], fb, cudaMemcpyDeviceToDevice, c->stream);
    cudaMemcpyAsync(save + fb, tmp->phi[p0], pb, cudaMemcpyDeviceToDevice, c->stream);
    cudaMemcpyAsync(save + fb + pb, tmp->T[q0], pb, cudaMemcpyDeviceToDevice, c->stream);
    auto restore = [&]() {
        int r = lf::wait_stream(c->stream);
        if (r != LF_OK) return r;
        tmp->fcur = f0; tmp->pcur = p0; tmp->tcur = q0;
        *const_cast<int*>(tmp->flag_host) = 0;
        if (cudaMemcpyAsync(tmp->f[f0], save, fb, cudaMemcpyDeviceToDevice, c->stream) != cudaSuccess ||
            cudaMemcpyAsync(tmp->phi[p0], save + fb, pb, cudaMemcpyDeviceToDevice, c->stream) != cudaSuccess ||
            cudaMemcpyAsync(tmp->T[q0], save + fb + pb, pb, cudaMemcpyDeviceToDevice, c->stream) != cudaSuccess)
            return (int)LF_ECUDA;
        return (int)LF_OK;
    };
    cudaEvent_t t0, t1;
    if (cudaEventCreate(&t0) != cudaSuccess || cudaEventCreate(&t1) != cudaSuccess) {
        cudaFree(save);
        lf_destroy(tmp);
        return LF_ECUDA;
    }
    const std::vector<std::pair<int, int>> cand = candidates(c);
    Choice best{cand[0].first, cand[0].second, 1e30f, (int)cand.size()};
    for (const auto& vp : cand) {
        if ((rc = restore()) != LF_OK) break;
        lf_set_kernel_variant(tmp, vp.first, vp.second);
        if ((rc = lf_step(tmp, 2)) != LF_OK) break;       // warm: first launch, attributes, caches
        cudaEventRecord(t0, c->stream);
        rc = lf_step(tmp, reps);
        cudaEventRecord(t1, c->stream);
        if (rc == LF_ENONFINITE) {                          // the timed steps were not all launched
            rc = LF_OK;
            continue;
        }
        if (rc != LF_OK || (rc = lf::wait_stream(c->stream)) != LF_OK) break;
        if (*tmp->flag_host) continue;                      // a trial state went non-finite: not timed
        float ms = 0;
        cudaEventElapsedTime(&ms, t0, t1);
        ms /= reps;
        if (ms < best.ms) { best.ms = ms; best.variant = vp.first; best.param = vp.second; }
    }
    cudaEventDestroy(t0);
    cudaEventDestroy(t1);
    if (rc == LF_OK) rc = lf::wait_stream(c->stream);
    cudaFree(save);
    lf_destroy(tmp);
    if (rc != LF_OK) return rc;
    {
        std::lock_guard<std::mutex> lock(g_mu);
        g_cache[key] = best;
    }
    c->g.variant = best.variant;
    c->g.tune = best.param;
    if (variant) *variant = best.variant;
    if (param) *param = best.param;
    if (ms_per_step) *ms_per_step = best.ms;
    return LF_OK;
}
