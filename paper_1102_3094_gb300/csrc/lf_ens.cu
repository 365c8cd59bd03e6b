// lf_ens.cu -- batched ensembles of independent 2D FP32 runs (include/lf_ens.h).
//
// Every run is an ordinary context placed in one shared device arena.  A time
// step of the whole ensemble is one launch of a persistent kernel that walks
// a work list of (run, strip, pair) items -- each item is exactly the
// two-lane row-marching step of lf_march2d_x2.cuh (two segments of a strip
// marching away from their common row) -- followed, when some runs need extra
// temperature sub-steps, by one launch per sub-step over the tiles of those
// runs.  Runs with the isotropic stencils are (run, strip, pair) items of a
// second persistent kernel that runs the two-lane isotropic row march
// (lf_march2d_iso.cuh), the code a single isotropic FP32 run uses by default.
// Every run returns to its starting buffers
// after two steps (f and phi flip once per step, T flips nsub times), so two
// steps are captured in one CUDA graph and replayed; single-step graphs handle
// odd counts.
#include <algorithm>
#include <cmath>
#include <cstdlib>
#include <cstring>
#include <map>
#include <tuple>
#include <new>
#include <utility>
#include <vector>

#include "lf_ctx.cuh"
#include "lf_ens.h"
#include "lf_march2d_iso.cuh"
#include "lf_march2d_x2.cuh"
#include "lf_tile2d.cuh"

using namespace lf;

namespace {

// Strips of 56 columns (64-thread CTAs) leave less idle width on 128^2 ..
// 512^2 lattices; 120-column strips (128 threads) issue fewer halo columns on
// wide ones.  The tuner picks per lattice size.
constexpr int kD = 3;
template <int NT>
using MarchCfg = march::March2<NT, kD>;
template <int NT>
using IsoCfg = march::MarchIso2<NT, kD>;

struct EnsRun {
    Geom g;
    Phys<float> p;
    StepIO<float> io;
};

struct EnsItem {
    int run, strip, pair, npairs;
};

struct EnsT {
    Geom g;
    Phys<float> p;
    const float* Tin;
    float* Tout;
};

struct EnsTItem {
    int run, bx, by;
};

// Isotropic runs: (run, strip, pair) items of the two-lane isotropic march,
// with the launch bounds of the single-run kernel, so both compile the same
// step.
template <int NT, int MINB>
__global__ void __launch_bounds__(NT, MINB) k_ens_march2d_iso(const EnsRun* __restrict__ runs,
                                                             const EnsItem* __restrict__ items, int nitems)
{
    extern __shared__ __align__(16) unsigned char smem_raw[];
    for (int it = blockIdx.x; it < nitems; it += gridDim.x) {
        const EnsItem w = items[it];
        const EnsRun r = runs[w.run];
        if (r.p.hydro)
            march::march2d_pair_iso<NT, kD, true>(r.g, r.p, r.io, w.strip, w.pair, w.npairs, smem_raw);
        else
            march::march2d_pair_iso<NT, kD, false>(r.g, r.p, r.io, w.strip, w.pair, w.npairs, smem_raw);
        __syncthreads();   // the next item reuses the shared rings
    }
}
constexpr auto kIso64 = k_ens_march2d_iso<64, 6>;
constexpr auto kIso128 = k_ens_march2d_iso<128, 3>;

template <int NT, int MINB>
__global__ void __launch_bounds__(NT, MINB) k_ens_march2d(const EnsRun* __restrict__ runs,
                                                         const EnsItem* __restrict__ items, int nitems)
{
    extern __shared__ __align__(16) unsigned char smem_raw[];
    for (int it = blockIdx.x; it < nitems; it += gridDim.x) {
        const EnsItem w = items[it];
        const EnsRun r = runs[w.run];
        if (r.p.hydro)
            march::march2d_pair<NT, kD, true>(r.g, r.p, r.io, w.strip, w.pair, w.npairs, smem_raw);
        else
            march::march2d_pair<NT, kD, false>(r.g, r.p, r.io, w.strip, w.pair, w.npairs, smem_raw);
        __syncthreads();   // the next item reuses the shared rings
    }
}
// the single-run launcher's instantiations: 64 threads at six CTAs per SM, 128 at three
constexpr auto kEns64 = k_ens_march2d<64, 6>;
constexpr auto kEns128 = k_ens_march2d<128, 3>;

// Pairs of segments of a run with H rows per segment (as the single-run
// launcher counts them, so a run stepped alone with the same H matches).
int pairs_for(int ny, int H)
{
    int np = (ny + 2 * H - 1) / (2 * H);
    if (np > ny / 2) np = ny / 2;
    return np < 1 ? 1 : np;
}

__global__ void __launch_bounds__(256) k_ens_tsub2d(const EnsT* __restrict__ runs, const EnsTItem* __restrict__ items,
                                                   int nitems)
{
    for (int it = blockIdx.x; it < nitems; it += gridDim.x) {
        const EnsTItem w = items[it];
        const EnsT r = runs[w.run];
        const int x = w.bx * 32 + (threadIdx.x & 31), y = w.by * 8 + (threadIdx.x >> 5);
        if (x < r.g.nx && y < r.g.ny) {
            if (r.g.stencil == LF_STENCIL_ISOTROPIC) tile::tsub2d_site_iso(r.g, r.p, r.Tin, r.Tout, x, y);
            else march::tsub2d_site(r.g, r.p, r.Tin, r.Tout, x, y);
        }
    }
}

Phys<float> phys_f(const lf_ctx* c)
{
    const lf_params& p = c->params;
    Phys<float> ph;
    ph.b = (float)p.b; ph.kappa = (float)p.kappa; ph.c = (float)p.c; ph.Gamma = (float)p.Gamma; ph.Tc = (float)p.Tc;
    ph.T_w = (float)c->walls.T_w;
    ph.inv_Tc = (float)(1.0 / p.Tc);
    ph.t_update = !(std::isinf(p.xi) || p.xi == 0.0);
    ph.dxi = ph.t_update ? (float)(p.xi / c->nsub) : 0.f;
    ph.inv_tau = (float)(1.0 / p.tau);
    ph.guo = (float)(1.0 - 1.0 / (2.0 * p.tau));
    ph.n0 = (float)p.n0;
    ph.hydro = p.hydro;
    return ph;
}

struct Cursor {
    int f, p, t;
};

}  // namespace

struct lf_ens {
    int nruns;
    std::vector<lf_ctx*> runs;
    std::vector<int> rows;          // rows per segment (lane) per run
    std::vector<int> width;         // threads per march CTA per run: 64 (56 columns) or 128 (120)
    std::vector<char> active;       // 0 once lf_ens_prune retired the run (non-finite state)
    cudaStream_t stream;
    bool own_stream;
    unsigned char* arena;
    unsigned char* tables;          // device copies of the descriptor tables and work lists
    cudaGraphExec_t gA, gB, gAB;
    int parity;                     // 0: the next step is step A of the cycle, 1: step B
    std::vector<Cursor> base;       // buffer cursors at the start of step A
    int march_blocks[4];            // 64- and 128-thread march kernels, compact then isotropic
    int nitems[4];
    EnsItem* d_items[4];
};

namespace {

void free_graphs(lf_ens* e)
{
    if (e->gA) cudaGraphExecDestroy(e->gA);
    if (e->gB) cudaGraphExecDestroy(e->gB);
    if (e->gAB) cudaGraphExecDestroy(e->gAB);
    e->gA = e->gB = e->gAB = nullptr;
    if (e->tables) cudaFree(e->tables);
    e->tables = nullptr;
}

// Device layout of one half-cycle (step A or B): run table, T tables.
struct Half {
    EnsRun* runs;
    std::vector<EnsT*> ts;          // per extra sub-step s = 1 .. max_nsub - 1
};

int capture(lf_ens* e, const std::vector<int>& halves, const Half* H, const std::vector<EnsTItem*>& titems,
            const std::vector<int>& ntitems, cudaGraphExec_t* out)
{
    cudaGraph_t graph;
    if (cudaStreamBeginCapture(e->stream, cudaStreamCaptureModeThreadLocal) != cudaSuccess) return LF_ECUDA;
    for (int h : halves) {
        if (e->nitems[0] > 0)
            kEns64<<<e->march_blocks[0], 64, MarchCfg<64>::BYTES, e->stream>>>(H[h].runs, e->d_items[0], e->nitems[0]);
        if (e->nitems[1] > 0)
            kEns128<<<e->march_blocks[1], 128, MarchCfg<128>::BYTES, e->stream>>>(H[h].runs, e->d_items[1],
                                                                               e->nitems[1]);
        if (e->nitems[2] > 0)
            kIso64<<<e->march_blocks[2], 64, IsoCfg<64>::BYTES, e->stream>>>(H[h].runs, e->d_items[2], e->nitems[2]);
        if (e->nitems[3] > 0)
            kIso128<<<e->march_blocks[3], 128, IsoCfg<128>::BYTES, e->stream>>>(H[h].runs, e->d_items[3],
                                                                              e->nitems[3]);
        for (size_t s = 0; s < H[h].ts.size(); ++s) {
            if (ntitems[s] == 0) continue;
            const int blocks = std::min(ntitems[s], 152 * 8);
            k_ens_tsub2d<<<blocks, 256, 0, e->stream>>>(H[h].ts[s], titems[s], ntitems[s]);
        }
    }
    cudaError_t err = cudaStreamEndCapture(e->stream, &graph);
    if (err != cudaSuccess) return LF_ECUDA;
    err = cudaGraphInstantiate(out, graph, 0);
    cudaGraphDestroy(graph);
    return err == cudaSuccess ? LF_OK : LF_ECUDA;
}

// (Re)builds the descriptor tables, the work lists and the three graphs from
// the runs' current buffer cursors.
int build(lf_ens* e)
{
    free_graphs(e);
    const int R = e->nruns;
    int max_nsub = 1;
    for (lf_ctx* c : e->runs)
        if (phys_f(c).t_update) max_nsub = std::max(max_nsub, c->nsub);

    // host tables for both halves
    e->base.resize(R);
    std::vector<EnsRun> hr[2];
    std::vector<std::vector<EnsT>> ht[2];
    for (int h = 0; h < 2; ++h) {
        hr[h].resize(R);
        ht[h].assign(max_nsub - 1, std::vector<EnsT>(R));
    }
    for (int r = 0; r < R; ++r) {
        lf_ctx* c = e->runs[r];
        Cursor cur{c->fcur, c->pcur, c->tcur};
        e->base[r] = cur;
        const Phys<float> ph = phys_f(c);
        for (int h = 0; h < 2; ++h) {
            EnsRun& d = hr[h][r];
            std::memset(&d, 0, sizeof(d));
            d.g = c->g;
            d.p = ph;
            d.io.f_in = (const float*)c->f[cur.f];
            d.io.f_out = (float*)c->f[cur.f ^ 1];
            d.io.phi_in = (const float*)c->phi[cur.p];
            d.io.phi_out = (float*)c->phi[cur.p ^ 1];
            d.io.T_in = (const float*)c->T[cur.t];
            d.io.T_out = (float*)c->T[cur.t ^ 1];
            d.io.flag = c->flag_dev;
            if (c->params.hydro) cur.f ^= 1;
            cur.p ^= 1;
            cur.t ^= 1;
            for (int s = 1; s < max_nsub; ++s) {
                EnsT& t = ht[h][s - 1][r];
                t.g = c->g;
                t.p = ph;
                t.Tin = (const float*)c->T[cur.t];
                t.Tout = (float*)c->T[cur.t ^ 1];
                if (ph.t_update && s < c->nsub) cur.t ^= 1;
            }
        }
    }
    // work lists: march items per kind and CTA width (compact 64, 128,
    // isotropic 64, 128) sorted by cost (longest lane first), T tiles per
    // sub-step
    std::vector<EnsItem> items[4];
    for (int r = 0; r < R; ++r) {
        const lf_ctx* c = e->runs[r];
        if (!e->active[r]) continue;
        const bool iso = c->g.stencil == LF_STENCIL_ISOTROPIC;
        const int np = pairs_for(c->g.ny, e->rows[r]);
        const int wi = (e->width[r] == 64 ? 0 : 1) + (iso ? 2 : 0);
        const int U = (wi & 1) == 0 ? MarchCfg<64>::U : MarchCfg<128>::U;   // 56 or 120 columns for both kinds
        const int strips = (c->g.nx + U - 1) / U;
        for (int pr = 0; pr < np; ++pr)
            for (int st = 0; st < strips; ++st) items[wi].push_back({r, st, pr, np});
    }
    auto lane = [&](const EnsItem& w) {
        const int ny = e->runs[w.run]->g.ny;
        return (ny + 2 * w.npairs - 1) / (2 * w.npairs);
    };
    for (auto& it : items)
        std::stable_sort(it.begin(), it.end(), [&](const EnsItem& a, const EnsItem& b) { return lane(a) > lane(b); });
    std::vector<std::vector<EnsTItem>> titems(max_nsub > 1 ? max_nsub - 1 : 0);
    for (int s = 1; s < max_nsub; ++s)
        for (int r = 0; r < R; ++r) {
            const lf_ctx* c = e->runs[r];
            if (!e->active[r] || !phys_f(c).t_update || s >= c->nsub) continue;
            for (int by = 0; by < (c->g.ny + 7) / 8; ++by)
                for (int bx = 0; bx < (c->g.nx + 31) / 32; ++bx) titems[s - 1].push_back({r, bx, by});
        }
    // one device block for everything
    auto a256 = [](size_t v) { return (v + 255) / 256 * 256; };
    size_t bytes = 2 * a256(sizeof(EnsRun) * R);
    for (const auto& it : items) bytes += a256(sizeof(EnsItem) * it.size());
    for (int s = 1; s < max_nsub; ++s) bytes += 2 * a256(sizeof(EnsT) * R) + a256(sizeof(EnsTItem) * titems[s - 1].size());
    if (cudaMalloc((void**)&e->tables, bytes) != cudaSuccess) { cudaGetLastError(); return LF_ENOMEM; }
    unsigned char* p = e->tables;
    Half halves[2];
    std::vector<std::pair<void*, std::pair<const void*, size_t>>> copies;
    for (int h = 0; h < 2; ++h) {
        halves[h].runs = (EnsRun*)p;
        copies.push_back({p, {hr[h].data(), sizeof(EnsRun) * R}});
        p += a256(sizeof(EnsRun) * R);
    }
    for (int wi = 0; wi < 4; ++wi) {
        e->d_items[wi] = (EnsItem*)p;
        e->nitems[wi] = (int)items[wi].size();
        copies.push_back({p, {items[wi].data(), sizeof(EnsItem) * items[wi].size()}});
        p += a256(sizeof(EnsItem) * items[wi].size());
    }
    std::vector<EnsTItem*> d_titems;
    std::vector<int> ntitems;
    for (int s = 1; s < max_nsub; ++s) {
        for (int h = 0; h < 2; ++h) {
            halves[h].ts.push_back((EnsT*)p);
            copies.push_back({p, {ht[h][s - 1].data(), sizeof(EnsT) * R}});
            p += a256(sizeof(EnsT) * R);
        }
        d_titems.push_back((EnsTItem*)p);
        ntitems.push_back((int)titems[s - 1].size());
        copies.push_back({p, {titems[s - 1].data(), sizeof(EnsTItem) * titems[s - 1].size()}});
        p += a256(sizeof(EnsTItem) * titems[s - 1].size());
    }
    for (auto& cp : copies)
        if (cp.second.second && cudaMemcpyAsync(cp.first, cp.second.first, cp.second.second, cudaMemcpyHostToDevice,
                                                e->stream) != cudaSuccess)
            return LF_ECUDA;
    int rc = wait_stream(e->stream);   // host vectors go out of scope
    if (rc != LF_OK) return rc;

    if (cudaFuncSetAttribute(kEns64, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)MarchCfg<64>::BYTES) !=
            cudaSuccess ||
        cudaFuncSetAttribute(kEns128, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)MarchCfg<128>::BYTES) !=
            cudaSuccess ||
        cudaFuncSetAttribute(kIso64, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)IsoCfg<64>::BYTES) !=
            cudaSuccess ||
        cudaFuncSetAttribute(kIso128, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)IsoCfg<128>::BYTES) !=
            cudaSuccess)
        return LF_ECUDA;
    int per_sm[4] = {0, 0, 0, 0}, sms = 0, dev = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm[0], kEns64, 64, MarchCfg<64>::BYTES);
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm[1], kEns128, 128, MarchCfg<128>::BYTES);
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm[2], kIso64, 64, IsoCfg<64>::BYTES);
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm[3], kIso128, 128, IsoCfg<128>::BYTES);
    for (int wi = 0; wi < 4; ++wi)
        e->march_blocks[wi] = std::max(1, std::min(e->nitems[wi], std::max(1, per_sm[wi]) * std::max(1, sms)));

    if ((rc = capture(e, {0}, halves, d_titems, ntitems, &e->gA)) != LF_OK) return rc;
    if ((rc = capture(e, {1}, halves, d_titems, ntitems, &e->gB)) != LF_OK) return rc;
    if ((rc = capture(e, {0, 1}, halves, d_titems, ntitems, &e->gAB)) != LF_OK) return rc;
    e->parity = 0;
    return LF_OK;
}

void advance_cursors(lf_ens* e, int64_t n)
{
    for (size_t r = 0; r < e->runs.size(); ++r) {
        if (!e->active[r]) continue;
        lf_ctx* c = e->runs[r];
        const bool tu = phys_f(c).t_update;
        const int tflips = tu ? c->nsub : 1;
        if ((n & 1) != 0) {
            if (c->params.hydro) c->fcur ^= 1;
            c->pcur ^= 1;
            if (tflips & 1) c->tcur ^= 1;
        }
        c->step += n;
        c->aux_valid = false;
    }
}

}  // namespace

extern "C" {

int lf_ens_create(int nruns, const lf_grid* grids, const lf_walls* walls, const lf_params* params, void* stream,
                  lf_ens** out)
{
    if (!out || nruns < 1 || !grids || !walls || !params) return LF_EINVAL;
    *out = nullptr;
    std::vector<size_t> ws(nruns);
    size_t total = 0;
    for (int r = 0; r < nruns; ++r) {
        if (grids[r].d != 2 || params[r].precision != LF_FP32 || grids[r].ny < 2) return LF_EINVAL;
        lf_params p = params[r];
        p.workspace = nullptr;
        p.workspace_bytes = 0;
        int rc = lf_workspace_bytes(&grids[r], &walls[r], &p, &ws[r]);
        if (rc != LF_OK) return rc;
        total += (ws[r] + 255) / 256 * 256;
    }
    lf_ens* e = new (std::nothrow) lf_ens();
    if (!e) return LF_ENOMEM;
    e->nruns = nruns;
    e->stream = (cudaStream_t)stream;
    if (!e->stream) {
        if (cudaStreamCreateWithFlags(&e->stream, cudaStreamNonBlocking) != cudaSuccess) {
            delete e;
            return LF_ECUDA;
        }
        e->own_stream = true;
    }
    if (cudaMalloc((void**)&e->arena, total) != cudaSuccess) {
        cudaGetLastError();
        if (e->own_stream) cudaStreamDestroy(e->stream);
        delete e;
        return LF_ENOMEM;
    }
    size_t off = 0;
    int rc = LF_OK;
    for (int r = 0; r < nruns && rc == LF_OK; ++r) {
        lf_params p = params[r];
        p.stream = e->stream;
        p.workspace = e->arena + off;
        p.workspace_bytes = ws[r];
        off += (ws[r] + 255) / 256 * 256;
        lf_ctx* c = nullptr;
        rc = lf_create(&grids[r], &walls[r], &p, &c);
        if (rc == LF_OK) {
            c->ens_member = true;
            e->runs.push_back(c);
            e->rows.push_back(c->g.ny / 2 < 16 ? (c->g.ny / 2 > 0 ? c->g.ny / 2 : 1) : 16);
            e->width.push_back(64);
            e->active.push_back(1);
        }
    }
    if (rc == LF_OK) rc = build(e);
    if (rc != LF_OK) {
        lf_ens_destroy(e);
        return rc;
    }
    *out = e;
    return LF_OK;
}

int lf_ens_tune(lf_ens* e, int reps)
{
    if (!e || reps < 1) return LF_EINVAL;
    int rc = wait_stream(e->stream);
    if (rc != LF_OK) return rc;
    // A scratch ensemble of the same runs, so that every candidate is timed
    // as what it is for: the throughput of the whole batch, not the latency
    // of one run alone (which favours short segments and many CTAs).
    const int R = e->nruns;
    std::vector<lf_grid> G(R);
    std::vector<lf_walls> W(R);
    std::vector<lf_params> P(R);
    for (int r = 0; r < R; ++r) {
        G[r] = e->runs[r]->grid;
        W[r] = e->runs[r]->walls;
        P[r] = e->runs[r]->params;
    }
    lf_ens* sc = nullptr;
    if ((rc = lf_ens_create(R, G.data(), W.data(), P.data(), e->stream, &sc)) != LF_OK) return rc;
    sc->width = e->width;
    sc->rows = e->rows;
    sc->active = e->active;
    cudaEvent_t t0, t1;
    cudaEventCreate(&t0);
    cudaEventCreate(&t1);
    // one pass of coordinate descent over the (lattice size, stencil) classes
    // of the runs
    using Key = std::tuple<int, int, int>;
    std::vector<Key> keys;
    auto key_of = [&](const lf_ctx* c) { return Key{c->g.nx, c->g.ny, c->g.stencil}; };
    for (int r = 0; r < R; ++r) {
        if (!e->active[r]) continue;
        const Key key = key_of(e->runs[r]);
        if (std::find(keys.begin(), keys.end(), key) == keys.end()) keys.push_back(key);
    }
    auto set_shape = [&](lf_ens* x, const Key& key, int w, int h) {
        for (int r = 0; r < R; ++r)
            if (key_of(e->runs[r]) == key) {
                x->width[r] = w;
                x->rows[r] = h;
            }
    };
    const int cand[] = {1, 2, 3, 4, 6, 8, 12, 16, 24, 32, 48, 64, 96, 128};
    for (const auto& key : keys) {
        const int ny = std::get<1>(key);
        float best_ms = 1e30f;
        std::pair<int, int> best_wh{64, 16};
        for (int w : {64, 128})
            for (int h : cand) {
                if (2 * h > ny && h != cand[0]) continue;     // two segments of h rows per CTA
                set_shape(sc, key, w, h);
                if ((rc = build(sc)) != LF_OK) break;
                if ((rc = lf_ens_step(sc, 2)) != LF_OK) break;
                cudaEventRecord(t0, sc->stream);
                if ((rc = lf_ens_step(sc, reps)) != LF_OK) break;
                cudaEventRecord(t1, sc->stream);
                if ((rc = wait_stream(sc->stream)) != LF_OK) break;
                float ms = 0;
                cudaEventElapsedTime(&ms, t0, t1);
                if (ms < best_ms) { best_ms = ms; best_wh = {w, h}; }
            }
        if (rc != LF_OK) break;
        set_shape(sc, key, best_wh.first, best_wh.second);
    }
    cudaEventDestroy(t0);
    cudaEventDestroy(t1);
    if (rc == LF_OK) {
        e->width = sc->width;
        e->rows = sc->rows;
    }
    lf_ens_destroy(sc);
    if (rc != LF_OK) return rc;
    return build(e);
}

int lf_ens_rows(const lf_ens* e, int run)
{
    if (!e || run < 0 || run >= e->nruns) return LF_EINVAL;
    return e->rows[run];
}

int lf_ens_prune(lf_ens* e, int* nactive)
{
    if (!e) return LF_EINVAL;
    int rc = wait_stream(e->stream);
    if (rc != LF_OK) return rc;
    bool changed = false;
    int live = 0;
    for (int r = 0; r < e->nruns; ++r) {
        if (e->active[r] && e->runs[r]->flag_host && *e->runs[r]->flag_host) {
            e->active[r] = 0;
            changed = true;
        }
        live += e->active[r] ? 1 : 0;
    }
    // the two-step graphs assume every run starts step A of a cycle: a
    // rebuild restarts the cycle from the runs' present buffers
    if (changed && (rc = build(e)) != LF_OK) return rc;
    if (nactive) *nactive = live;
    return LF_OK;
}

int lf_ens_active(const lf_ens* e, int run)
{
    if (!e || run < 0 || run >= e->nruns) return LF_EINVAL;
    return e->active[run] ? 1 : 0;
}

int lf_ens_param(const lf_ens* e, int run)
{
    if (!e || run < 0 || run >= e->nruns) return LF_EINVAL;
    return (e->width[run] == 64 ? 1 << 16 : 0) | e->rows[run];
}

int lf_ens_step(lf_ens* e, int64_t nsteps)
{
    lf::NvtxRange nvtx_range("lf_ens_step");
    if (!e || nsteps < 0) return LF_EINVAL;
    if (cudaGetLastError() != cudaSuccess) return LF_ECUDA;
    int64_t n = nsteps;
    while (n > 0) {
        cudaGraphExec_t g;
        int64_t k;
        if (e->parity == 1) { g = e->gB; k = 1; }
        else if (n >= 2) { g = e->gAB; k = 2; }
        else { g = e->gA; k = 1; }
        if (cudaGraphLaunch(g, e->stream) != cudaSuccess) return LF_ECUDA;
        e->parity = (int)((e->parity + k) & 1);
        n -= k;
    }
    advance_cursors(e, nsteps);
    return LF_OK;
}

int lf_ens_run(lf_ens* e, int run, lf_ctx** ctx)
{
    if (!e || !ctx || run < 0 || run >= e->nruns) return LF_EINVAL;
    *ctx = e->runs[run];
    return LF_OK;
}

int lf_ens_sync(lf_ens* e)
{
    if (!e) return LF_EINVAL;
    return wait_stream(e->stream);
}

void lf_ens_destroy(lf_ens* e)
{
    if (!e) return;
    if (e->stream) wait_stream(e->stream);
    free_graphs(e);
    for (lf_ctx* c : e->runs) lf_destroy(c);
    if (e->arena) cudaFree(e->arena);
    if (e->own_stream) cudaStreamDestroy(e->stream);
    cudaGetLastError();
    delete e;
}

}  // extern "C"
