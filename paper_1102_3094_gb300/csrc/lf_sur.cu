// lf_sur.cu -- the learned surrogate of include/lf_sur.h: parameters, forward
// and backward passes built from the tensor-core convolutions of
// lf_sur_conv.cu, MSE loss, Adam with FP32 master weights, and the run that
// interleaves surrogate windows with plain steps of a context, with a plain
// shadow window as check and fallback.
#include <cuda_bf16.h>

#include <algorithm>
#include <cmath>
#include <cstdlib>
#include <cstring>
#include <new>
#include <vector>

#include "lf_ctx.cuh"
#include "lf_sur.h"

using namespace lf;

namespace {

constexpr int kLayers = 6;
constexpr int kCin[kLayers] = {16, 64, 64, 64, 64, 64};
constexpr int kCout[kLayers] = {64, 64, 64, 64, 64, 16};

size_t wcount(int l) { return (size_t)9 * kCout[l] * kCin[l]; }

uint64_t splitmix(uint64_t& s)
{
    uint64_t z = (s += 0x9E3779B97F4A7C15ull);
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
    return z ^ (z >> 31);
}

// ---- small kernels ----------------------------------------------------------

// raw fields [B][4][NY][NX] (phi, T, ux, uy) -> x16 padded NHWC BF16 (channels
// 4..15 zero, halo per the lattice) and x4 = normalised FP32 [B][NY][NX][4]
__global__ void k_norm_in(const float* __restrict__ raw, int B, int NY, int NX, lf_sur_norm nm,
                          __nv_bfloat16* __restrict__ x16, float* __restrict__ x4)
{
    const int64_t N = (int64_t)B * NY * NX;
    for (int64_t k = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; k < N; k += (int64_t)gridDim.x * blockDim.x) {
        const int x = (int)(k % NX);
        const int64_t r = k / NX;
        const int y = (int)(r % NY), b = (int)(r / NY);
        __align__(16) __nv_bfloat16 v[16];
#pragma unroll
        for (int c = 0; c < 16; ++c) v[c] = __float2bfloat16_rn(0.f);
#pragma unroll
        for (int c = 0; c < 4; ++c) {
            const float s = (raw[(((int64_t)b * 4 + c) * NY + y) * NX + x] - (float)nm.offset[c]) * (float)(1.0 / nm.scale[c]);
            x4[k * 4 + c] = s;
            v[c] = __float2bfloat16_rn(s);
        }
        const int64_t po = ((int64_t)b * (NY + 2) + y + 1) * (NX + 2) + x + 1;
        uint4* d = reinterpret_cast<uint4*>(x16 + po * 16);
        d[0] = reinterpret_cast<uint4*>(v)[0];
        d[1] = reinterpret_cast<uint4*>(v)[1];
        if (x == 0 || x == NX - 1) {
            const int64_t ph = ((int64_t)b * (NY + 2) + y + 1) * (NX + 2) + (x == 0 ? NX + 1 : 0);
            uint4* dh = reinterpret_cast<uint4*>(x16 + ph * 16);
            dh[0] = reinterpret_cast<uint4*>(v)[0];
            dh[1] = reinterpret_cast<uint4*>(v)[1];
        }
    }
}

__global__ void k_norm_target(const float* __restrict__ raw, int B, int NY, int NX, lf_sur_norm nm, float* __restrict__ t4)
{
    const int64_t N = (int64_t)B * NY * NX;
    for (int64_t k = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; k < N; k += (int64_t)gridDim.x * blockDim.x) {
        const int x = (int)(k % NX);
        const int64_t r = k / NX;
        const int y = (int)(r % NY), b = (int)(r / NY);
#pragma unroll
        for (int c = 0; c < 4; ++c)
            t4[k * 4 + c] = (raw[(((int64_t)b * 4 + c) * NY + y) * NX + x] - (float)nm.offset[c]) * (float)(1.0 / nm.scale[c]);
    }
}

__global__ void k_denorm(const float* __restrict__ y4, int B, int NY, int NX, lf_sur_norm nm, float* __restrict__ raw)
{
    const int64_t N = (int64_t)B * NY * NX;
    for (int64_t k = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; k < N; k += (int64_t)gridDim.x * blockDim.x) {
        const int x = (int)(k % NX);
        const int64_t r = k / NX;
        const int y = (int)(r % NY), b = (int)(r / NY);
#pragma unroll
        for (int c = 0; c < 4; ++c)
            raw[(((int64_t)b * 4 + c) * NY + y) * NX + x] = y4[k * 4 + c] * (float)nm.scale[c] + (float)nm.offset[c];
    }
}

// MSE over B NY NX 4 outputs: per-block FP64 partial of sum (y - t)^2, and the
// gradient g = 2 (y - t) / count into the padded 16-channel BF16 tensor
__global__ void k_mse(const float* __restrict__ y4, const float* __restrict__ t4, int B, int NY, int NX,
                      double* __restrict__ part, __nv_bfloat16* __restrict__ g16)
{
    __shared__ double red[256];
    const int64_t N = (int64_t)B * NY * NX;
    const float inv = (float)(2.0 / (4.0 * (double)N));
    double acc = 0.0;
    for (int64_t k = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; k < N; k += (int64_t)gridDim.x * blockDim.x) {
        const int x = (int)(k % NX);
        const int64_t r = k / NX;
        const int y = (int)(r % NY), b = (int)(r / NY);
        __align__(16) __nv_bfloat16 v[16];
#pragma unroll
        for (int c = 0; c < 16; ++c) v[c] = __float2bfloat16_rn(0.f);
#pragma unroll
        for (int c = 0; c < 4; ++c) {
            const float d = y4[k * 4 + c] - t4[k * 4 + c];
            acc += (double)d * d;
            v[c] = __float2bfloat16_rn(inv * d);
        }
        if (g16) {
            const int64_t po = ((int64_t)b * (NY + 2) + y + 1) * (NX + 2) + x + 1;
            uint4* dd = reinterpret_cast<uint4*>(g16 + po * 16);
            dd[0] = reinterpret_cast<uint4*>(v)[0];
            dd[1] = reinterpret_cast<uint4*>(v)[1];
            if (x == 0 || x == NX - 1) {
                const int64_t ph = ((int64_t)b * (NY + 2) + y + 1) * (NX + 2) + (x == 0 ? NX + 1 : 0);
                uint4* dh = reinterpret_cast<uint4*>(g16 + ph * 16);
                dh[0] = reinterpret_cast<uint4*>(v)[0];
                dh[1] = reinterpret_cast<uint4*>(v)[1];
            }
        }
    }
    red[threadIdx.x] = acc;
    __syncthreads();
    for (int s = 128; s > 0; s >>= 1) {
        if ((int)threadIdx.x < s) red[threadIdx.x] += red[threadIdx.x + s];
        __syncthreads();
    }
    if (threadIdx.x == 0) part[blockIdx.x] = red[0];
}

// bias gradient: db[o] = sum over interior pixels of g[p][o] (FP32 block sums, atomics)
__global__ void k_bias_grad(const __nv_bfloat16* __restrict__ g, int C, int B, int NY, int NX, float* __restrict__ db)
{
    const int o = threadIdx.x % C, lanes = blockDim.x / C;
    const int sub = threadIdx.x / C;
    const int64_t N = (int64_t)B * NY * NX;
    float acc = 0.f;
    for (int64_t k = (int64_t)blockIdx.x * lanes + sub; k < N; k += (int64_t)gridDim.x * lanes) {
        const int x = (int)(k % NX);
        const int64_t r = k / NX;
        const int y = (int)(r % NY), b = (int)(r / NY);
        const int64_t po = ((int64_t)b * (NY + 2) + y + 1) * (NX + 2) + x + 1;
        acc += __bfloat162float(g[po * C + o]);
    }
    atomicAdd(&db[o], acc);
}

// Adam on FP32 master parameters; writes the BF16 weights for the forward pass
// and the tap-flipped, transposed BF16 copies for the backward data pass.
struct AdamLayer {
    float* w; float* m; float* v; const float* gw;
    float* b; float* mb; float* vb; const float* gb;
    __nv_bfloat16* wbf; __nv_bfloat16* wtbf;
    int cin, cout;
};

// Squared norm of one layer's gradients (weights and biases) added to *acc.
__global__ void k_grad_sumsq(const float* __restrict__ gw, int nw, const float* __restrict__ gb, int nb, double* acc)
{
    double v = 0.0;
    for (int k = blockIdx.x * blockDim.x + threadIdx.x; k < nw + nb; k += gridDim.x * blockDim.x) {
        const double g = k < nw ? gw[k] : gb[k - nw];
        v += g * g;
    }
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    if ((threadIdx.x & 31) == 0) atomicAdd(acc, v);
}

// Adam with the gradients scaled by min(1, clip / ||g||) (global norm
// clipping; clip = 0 leaves them as they are).
__global__ void k_adam(AdamLayer L, float lr, float b1, float b2, float eps, float c1, float c2, int do_update,
                       const double* gnorm2, float clip)
{
    const int nw = 9 * L.cout * L.cin;
    float gs = 1.f;
    if (do_update && clip > 0.f) {
        const double n = sqrt(*gnorm2);
        if (n > (double)clip) gs = (float)((double)clip / n);
    }
    for (int k = blockIdx.x * blockDim.x + threadIdx.x; k < nw + L.cout; k += gridDim.x * blockDim.x) {
        if (k < nw) {
            float w = L.w[k];
            if (do_update) {
                const float g = gs * L.gw[k];
                const float m = b1 * L.m[k] + (1.f - b1) * g, v = b2 * L.v[k] + (1.f - b2) * g * g;
                L.m[k] = m;
                L.v[k] = v;
                w -= lr * (m * c1) / (sqrtf(v * c2) + eps);
                L.w[k] = w;
            }
            const int t = k / (L.cout * L.cin), rem = k - t * L.cout * L.cin;
            const int o = rem / L.cin, i = rem - o * L.cin;
            const __nv_bfloat16 wb = __float2bfloat16_rn(w);
            L.wbf[k] = wb;
            L.wtbf[((int64_t)(8 - t) * L.cin + i) * L.cout + o] = wb;    // W'[8-t][i][o] = W[t][o][i]
        } else if (do_update) {
            const int o = k - nw;
            const float g = gs * L.gb[o];
            const float m = b1 * L.mb[o] + (1.f - b1) * g, v = b2 * L.vb[o] + (1.f - b2) * g * g;
            L.mb[o] = m;
            L.vb[o] = v;
            L.b[o] -= lr * (m * c1) / (sqrtf(v * c2) + eps);
        }
    }
}

unsigned blocks_for(int64_t n)
{
    int64_t b = (n + 255) / 256;
    return (unsigned)std::max<int64_t>(1, std::min<int64_t>(b, 152 * 8));
}

}  // namespace

struct lf_sur {
    int NY, NX, maxB;
    lf_sur_norm norm;
    cudaStream_t stream;
    unsigned char* block;        // one device allocation for everything below
    size_t bytes;
    // parameters (FP32 master), Adam moments, gradients; BF16 copies
    float* w[kLayers]; float* m[kLayers]; float* v[kLayers]; float* gw[kLayers];
    float* b[kLayers]; float* mb[kLayers]; float* vb[kLayers]; float* gb[kLayers];
    __nv_bfloat16* wbf[kLayers]; __nv_bfloat16* wtbf[kLayers];
    // activations (padded NHWC BF16)
    __nv_bfloat16* x16;          // input
    __nv_bfloat16* h[kLayers - 1];   // h1 .. h5 (64 ch)
    __nv_bfloat16* z[kLayers - 1];   // z1 .. z5 (pre-activations, masks)
    __nv_bfloat16* g16;          // dL/dz6 (16 ch)
    __nv_bfloat16* ga; __nv_bfloat16* gb2; __nv_bfloat16* gz;   // dL/dh ping-pong and dL/dz (64 ch)
    __nv_bfloat16* gz_alt;
    float* x4; float* y4; float* t4;
    float* part;                 // weight-gradient partials
    size_t part_floats;
    double* loss_part;           // k_mse block partials
    int* err;
    int step;                    // Adam step count
    double* gnorm2;              // squared global gradient norm of the last step
    float clip;                  // largest global gradient norm Adam sees (0 = no clipping)
};

namespace {

int sync_check(lf_sur* s)
{
    int rc = wait_stream(s->stream);
    if (rc != LF_OK) return rc;
    int e = 0;
    if (cudaMemcpy(&e, s->err, sizeof(int), cudaMemcpyDeviceToHost) != cudaSuccess) return LF_ECUDA;
    return e ? LF_ETIMEOUT : LF_OK;
}

int refresh_bf16(lf_sur* s, int do_update, float lr)
{
    s->step += do_update ? 1 : 0;
    const float b1 = 0.9f, b2 = 0.999f, eps = 1e-8f;
    const float c1 = do_update ? (float)(1.0 / (1.0 - std::pow(b1, s->step))) : 1.f;
    const float c2 = do_update ? (float)(1.0 / (1.0 - std::pow(b2, s->step))) : 1.f;
    if (do_update) {
        if (cudaMemsetAsync(s->gnorm2, 0, sizeof(double), s->stream) != cudaSuccess) return LF_ECUDA;
        for (int l = 0; l < kLayers; ++l)
            k_grad_sumsq<<<64, 256, 0, s->stream>>>(s->gw[l], (int)wcount(l), s->gb[l], kCout[l], s->gnorm2);
    }
    for (int l = 0; l < kLayers; ++l) {
        AdamLayer L{s->w[l], s->m[l], s->v[l], s->gw[l], s->b[l], s->mb[l], s->vb[l], s->gb[l], s->wbf[l], s->wtbf[l],
                    kCin[l], kCout[l]};
        k_adam<<<blocks_for((int64_t)wcount(l) + kCout[l]), 256, 0, s->stream>>>(L, lr, b1, b2, eps, c1, c2, do_update,
                                                                               s->gnorm2, s->clip);
    }
    return cudaGetLastError() == cudaSuccess ? LF_OK : LF_ECUDA;
}

// keep_z: store each layer's pre-activation values for the backward pass
// (training); a prediction does not need them
int forward(lf_sur* s, const float* raw, int B, bool keep_z)
{
    const int NY = s->NY, NX = s->NX;
    const int64_t N = (int64_t)B * NY * NX;
    k_norm_in<<<blocks_for(N), 256, 0, s->stream>>>(raw, B, NY, NX, s->norm, s->x16, s->x4);
    int rc = lf_sur_conv3x3(B, NY, NX, 16, 64, s->x16, s->wbf[0], s->b[0], 1, nullptr, nullptr, s->h[0], nullptr,
                            keep_z ? s->z[0] : nullptr, nullptr, nullptr, s->err, s->stream);
    for (int l = 1; l < 5 && rc == LF_OK; ++l)
        rc = lf_sur_conv3x3(B, NY, NX, 64, 64, s->h[l - 1], s->wbf[l], s->b[l], 1, s->h[l - 1], nullptr, s->h[l],
                            nullptr, keep_z ? s->z[l] : nullptr, nullptr, nullptr, s->err, s->stream);
    if (rc == LF_OK)
        rc = lf_sur_conv3x3(B, NY, NX, 64, 16, s->h[4], s->wbf[5], s->b[5], 0, nullptr, nullptr, nullptr, nullptr,
                            nullptr, s->x4, s->y4, s->err, s->stream);
    return rc;
}

// loss (host, FP64) and, when grads, every gradient into gw / gb
int loss_and_grads(lf_sur* s, const float* x, const float* y, int B, double* loss, bool grads)
{
    const int NY = s->NY, NX = s->NX;
    const int64_t N = (int64_t)B * NY * NX;
    int rc = forward(s, x, B, grads);
    if (rc != LF_OK) return rc;
    k_norm_target<<<blocks_for(N), 256, 0, s->stream>>>(y, B, NY, NX, s->norm, s->t4);
    const unsigned mb = blocks_for(N);
    k_mse<<<mb, 256, 0, s->stream>>>(s->y4, s->t4, B, NY, NX, s->loss_part, grads ? s->g16 : nullptr);
    if (grads) {
        for (int l = 0; l < kLayers; ++l) cudaMemsetAsync(s->gb[l], 0, sizeof(float) * kCout[l], s->stream);
        // layer 6: dW6 from h5 and g16; dL/dh5 = conv(g16, W6'), mask by z5 -> dL/dz5
        const __nv_bfloat16* hin[kLayers] = {s->x16, s->h[0], s->h[1], s->h[2], s->h[3], s->h[4]};
        rc = lf_sur_conv3x3_wgrad(B, NY, NX, 64, 16, s->h[4], s->g16, s->part, s->part_floats, s->gw[5], s->err,
                                  s->stream);
        k_bias_grad<<<304, 256, 0, s->stream>>>(s->g16, 16, B, NY, NX, s->gb[5]);
        __nv_bfloat16* gh = s->ga;       // dL/dh_l
        __nv_bfloat16* gz = s->gz;       // dL/dz_l
        if (rc == LF_OK)
            rc = lf_sur_conv3x3(B, NY, NX, 16, 64, s->g16, s->wtbf[5], nullptr, 0, nullptr, s->z[4], gh, gz, nullptr,
                                nullptr, nullptr, s->err, s->stream);
        // layers 5 .. 2: dW_l from h_{l-1} and dL/dz_l; dL/dh_{l-1} = dL/dh_l + conv(dL/dz_l, W_l')
        for (int l = 4; l >= 1 && rc == LF_OK; --l) {
            rc = lf_sur_conv3x3_wgrad(B, NY, NX, 64, 64, hin[l], gz, s->part, s->part_floats, s->gw[l], s->err,
                                      s->stream);
            k_bias_grad<<<304, 256, 0, s->stream>>>(gz, 64, B, NY, NX, s->gb[l]);
            __nv_bfloat16* gh_next = (gh == s->ga) ? s->gb2 : s->ga;
            __nv_bfloat16* gz_next = (gz == s->gz) ? s->gz_alt : s->gz;
            if (rc == LF_OK)
                rc = lf_sur_conv3x3(B, NY, NX, 64, 64, gz, s->wtbf[l], nullptr, 0, gh, s->z[l - 1], gh_next, gz_next,
                                    nullptr, nullptr, nullptr, s->err, s->stream);
            gh = gh_next;
            gz = gz_next;
        }
        // layer 1: dW1 from x16 and dL/dz1
        if (rc == LF_OK)
            rc = lf_sur_conv3x3_wgrad(B, NY, NX, 16, 64, s->x16, gz, s->part, s->part_floats, s->gw[0], s->err,
                                      s->stream);
        k_bias_grad<<<304, 256, 0, s->stream>>>(gz, 64, B, NY, NX, s->gb[0]);
    }
    if (rc != LF_OK) return rc;
    std::vector<double> lp(mb);
    if (cudaMemcpyAsync(lp.data(), s->loss_part, sizeof(double) * mb, cudaMemcpyDeviceToHost, s->stream) != cudaSuccess)
        return LF_ECUDA;
    rc = sync_check(s);
    if (rc != LF_OK) return rc;
    double acc = 0.0;
    for (double v : lp) acc += v;
    *loss = acc / (4.0 * (double)N);
    return LF_OK;
}

}  // namespace

extern "C" {

int lf_sur_create(int NY, int NX, int max_batch, uint64_t seed, const lf_sur_norm* norm, void* stream, lf_sur** out)
{
    if (!out || !norm || NY < 1 || NX < 128 || NX % 128 != 0 || max_batch < 1) return LF_EINVAL;
    for (int c = 0; c < 4; ++c)
        if (!(norm->scale[c] > 0) || !std::isfinite(norm->offset[c])) return LF_EINVAL;
    *out = nullptr;
    lf_sur* s = new (std::nothrow) lf_sur();
    if (!s) return LF_ENOMEM;
    s->NY = NY; s->NX = NX; s->maxB = max_batch; s->norm = *norm; s->stream = (cudaStream_t)stream;
    auto a256 = [](size_t v) { return (v + 255) / 256 * 256; };
    const size_t pad_px = (size_t)max_batch * (NY + 2) * (NX + 2);
    const size_t px = (size_t)max_batch * NY * NX;
    s->part_floats = std::max({lf_sur_wgrad_scratch_floats(16, 64), lf_sur_wgrad_scratch_floats(64, 64),
                               lf_sur_wgrad_scratch_floats(64, 16)});
    size_t bytes = 0;
    for (int l = 0; l < kLayers; ++l)
        bytes += 4 * a256(4 * wcount(l)) + 4 * a256(4 * (size_t)kCout[l]) + 2 * a256(2 * wcount(l));
    bytes += a256(2 * pad_px * 16) * 2 + a256(2 * pad_px * 64) * (2 * 5 + 4);
    bytes += 3 * a256(4 * px * 4) + a256(4 * s->part_floats) + a256(8 * 152 * 8) + 256 + 256;
    if (cudaMalloc((void**)&s->block, bytes) != cudaSuccess) {
        cudaGetLastError();
        delete s;
        return LF_ENOMEM;
    }
    s->bytes = bytes;
    unsigned char* p = s->block;
    auto take = [&](size_t n) { unsigned char* r = p; p += a256(n); return r; };
    for (int l = 0; l < kLayers; ++l) {
        s->w[l] = (float*)take(4 * wcount(l)); s->m[l] = (float*)take(4 * wcount(l));
        s->v[l] = (float*)take(4 * wcount(l)); s->gw[l] = (float*)take(4 * wcount(l));
        s->b[l] = (float*)take(4 * kCout[l]); s->mb[l] = (float*)take(4 * kCout[l]);
        s->vb[l] = (float*)take(4 * kCout[l]); s->gb[l] = (float*)take(4 * kCout[l]);
        s->wbf[l] = (__nv_bfloat16*)take(2 * wcount(l)); s->wtbf[l] = (__nv_bfloat16*)take(2 * wcount(l));
    }
    s->x16 = (__nv_bfloat16*)take(2 * pad_px * 16);
    s->g16 = (__nv_bfloat16*)take(2 * pad_px * 16);
    for (int l = 0; l < 5; ++l) s->h[l] = (__nv_bfloat16*)take(2 * pad_px * 64);
    for (int l = 0; l < 5; ++l) s->z[l] = (__nv_bfloat16*)take(2 * pad_px * 64);
    s->ga = (__nv_bfloat16*)take(2 * pad_px * 64);
    s->gb2 = (__nv_bfloat16*)take(2 * pad_px * 64);
    s->gz = (__nv_bfloat16*)take(2 * pad_px * 64);
    s->gz_alt = (__nv_bfloat16*)take(2 * pad_px * 64);
    s->x4 = (float*)take(4 * px * 4); s->y4 = (float*)take(4 * px * 4); s->t4 = (float*)take(4 * px * 4);
    s->part = (float*)take(4 * s->part_floats);
    s->loss_part = (double*)take(8 * 152 * 8);
    s->err = (int*)take(4);
    s->gnorm2 = (double*)take(8);
    s->clip = 1.0f;
    // zero everything (halo rows of the activations stay zero for good), then
    // He-uniform weights from SplitMix64, the last layer scaled down so the
    // untrained network starts close to the identity map
    int rc = cudaMemsetAsync(s->block, 0, bytes, s->stream) == cudaSuccess ? LF_OK : LF_ECUDA;
    uint64_t st = seed;
    for (int l = 0; l < kLayers && rc == LF_OK; ++l) {
        std::vector<float> hw(wcount(l));
        const double lim = std::sqrt(6.0 / (9.0 * (l == 0 ? 4 : kCin[l]))) * (l == kLayers - 1 ? 0.1 : 1.0);
        for (size_t k = 0; k < hw.size(); ++k) {
            const int i = (int)(k % kCin[l]);
            const double u = (double)(splitmix(st) >> 11) * 0x1.0p-53;
            hw[k] = (l == 0 && i >= 4) ? 0.f : (float)(lim * (2.0 * u - 1.0));
        }
        if (cudaMemcpyAsync(s->w[l], hw.data(), 4 * hw.size(), cudaMemcpyHostToDevice, s->stream) != cudaSuccess)
            rc = LF_ECUDA;
        if (rc == LF_OK) rc = wait_stream(s->stream);
    }
    if (rc == LF_OK) rc = refresh_bf16(s, 0, 0.f);
    if (rc == LF_OK) rc = sync_check(s);
    if (rc != LF_OK) {
        lf_sur_destroy(s);
        return rc;
    }
    *out = s;
    return LF_OK;
}

int lf_sur_set_clip(lf_sur* s, float max_norm)
{
    if (!s || !(max_norm >= 0.f)) return LF_EINVAL;
    s->clip = max_norm;
    return LF_OK;
}

size_t lf_sur_param_count(void)
{
    size_t n = 0;
    for (int l = 0; l < kLayers; ++l) n += wcount(l) + kCout[l];
    return n;
}

int lf_sur_get_params(lf_sur* s, float* host)
{
    if (!s || !host) return LF_EINVAL;
    size_t off = 0;
    for (int l = 0; l < kLayers; ++l) {
        if (cudaMemcpyAsync(host + off, s->w[l], 4 * wcount(l), cudaMemcpyDeviceToHost, s->stream) != cudaSuccess)
            return LF_ECUDA;
        off += wcount(l);
        if (cudaMemcpyAsync(host + off, s->b[l], 4 * kCout[l], cudaMemcpyDeviceToHost, s->stream) != cudaSuccess)
            return LF_ECUDA;
        off += kCout[l];
    }
    return wait_stream(s->stream);
}

int lf_sur_set_params(lf_sur* s, const float* host)
{
    if (!s || !host) return LF_EINVAL;
    size_t off = 0;
    for (int l = 0; l < kLayers; ++l) {
        if (cudaMemcpyAsync(s->w[l], host + off, 4 * wcount(l), cudaMemcpyHostToDevice, s->stream) != cudaSuccess)
            return LF_ECUDA;
        off += wcount(l);
        if (cudaMemcpyAsync(s->b[l], host + off, 4 * kCout[l], cudaMemcpyHostToDevice, s->stream) != cudaSuccess)
            return LF_ECUDA;
        off += kCout[l];
    }
    int rc = refresh_bf16(s, 0, 0.f);
    return rc == LF_OK ? sync_check(s) : rc;
}

int lf_sur_grads(lf_sur* s, const float* x, const float* y, int B, double* loss, float* grads_host)
{
    if (!s || !x || !y || !loss || B < 1 || B > s->maxB) return LF_EINVAL;
    int rc = loss_and_grads(s, x, y, B, loss, grads_host != nullptr);
    if (rc != LF_OK || !grads_host) return rc;
    size_t off = 0;
    for (int l = 0; l < kLayers; ++l) {
        if (cudaMemcpyAsync(grads_host + off, s->gw[l], 4 * wcount(l), cudaMemcpyDeviceToHost, s->stream) != cudaSuccess)
            return LF_ECUDA;
        off += wcount(l);
        if (cudaMemcpyAsync(grads_host + off, s->gb[l], 4 * kCout[l], cudaMemcpyDeviceToHost, s->stream) != cudaSuccess)
            return LF_ECUDA;
        off += kCout[l];
    }
    return sync_check(s);
}

int lf_sur_train_step(lf_sur* s, const float* x, const float* y, int B, float lr, double* loss)
{
    lf::NvtxRange nvtx_range("lf_sur_train_step");
    if (!s || !x || !y || !loss || B < 1 || B > s->maxB || !(lr > 0)) return LF_EINVAL;
    int rc = loss_and_grads(s, x, y, B, loss, true);
    if (rc == LF_OK) rc = refresh_bf16(s, 1, lr);
    return rc;
}

int lf_sur_predict(lf_sur* s, const float* x, float* y, int B)
{
    lf::NvtxRange nvtx_range("lf_sur_predict");
    if (!s || !x || !y || B < 1 || B > s->maxB) return LF_EINVAL;
    int rc = forward(s, x, B, false);
    if (rc != LF_OK) return rc;
    k_denorm<<<blocks_for((int64_t)B * s->NY * s->NX), 256, 0, s->stream>>>(s->y4, B, s->NY, s->NX, s->norm, y);
    return cudaGetLastError() == cudaSuccess ? LF_OK : LF_ECUDA;
}

void lf_sur_destroy(lf_sur* s)
{
    if (!s) return;
    wait_stream(s->stream);
    if (s->block) cudaFree(s->block);
    cudaGetLastError();
    delete s;
}

}  // extern "C"

// ===========================================================================
// Interleaved run: surrogate windows of K steps alternate with plain windows;
// a plain shadow window from the same state checks every shadow_every-th
// surrogate window and replaces its result when the error is too large.
// ===========================================================================
namespace {

// Hand a predicted velocity to the populations of a 2D FP32 context (stored
// as deviations f_i - w_i n0): the equilibrium part moves from the current
// velocity to the predicted one at the current density, the non-equilibrium
// part (not predicted) is kept:
//   f_i += w_i n (3 e.du + 4.5 ((e.u')^2 - (e.u)^2) - 1.5 (u'.u' - u.u)).
__global__ void k_shift_u2d(Geom g, float n0, const float* __restrict__ ux0, const float* __restrict__ uy0,
                            const float* __restrict__ ux1, const float* __restrict__ uy1, float* __restrict__ f)
{
    const int64_t N = (int64_t)g.nx * g.ny;
    for (int64_t k = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; k < N; k += (int64_t)gridDim.x * blockDim.x) {
        const int x = (int)(k % g.nx), y = (int)(k / g.nx);
        const int64_t site = (int64_t)y * g.pitch + x;
        float df[D2Q9::Q], dn = 0.f;
#pragma unroll
        for (int i = 0; i < D2Q9::Q; ++i) {
            df[i] = f[i * g.plane + site];
            dn += df[i];
        }
        const float n = n0 + dn;
        const float ax = ux0[k], ay = uy0[k], bx = ux1[k], by = uy1[k];
        const float du2 = (bx * bx + by * by) - (ax * ax + ay * ay);
#pragma unroll
        for (int i = 0; i < D2Q9::Q; ++i) {
            const float ex = (float)D2Q9::ex(i), ey = (float)D2Q9::ey(i);
            const float ea = ex * ax + ey * ay, eb = ex * bx + ey * by;
            f[i * g.plane + site] = df[i] + (float)D2Q9::w(i) * n * (3.f * (eb - ea) + 4.5f * (eb * eb - ea * ea) - 1.5f * du2);
        }
    }
}

// sum (a - b)^2 and sum b^2 (FP64) over n values: per-block partials
__global__ void k_l2_parts(const float* __restrict__ a, const float* __restrict__ b, int64_t n, double* __restrict__ part)
{
    __shared__ double r0[256], r1[256];
    double s0 = 0.0, s1 = 0.0;
    for (int64_t k = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; k < n; k += (int64_t)gridDim.x * blockDim.x) {
        const double d = (double)a[k] - (double)b[k];
        s0 += d * d;
        s1 += (double)b[k] * (double)b[k];
    }
    r0[threadIdx.x] = s0;
    r1[threadIdx.x] = s1;
    __syncthreads();
    for (int s = 128; s > 0; s >>= 1) {
        if ((int)threadIdx.x < s) { r0[threadIdx.x] += r0[threadIdx.x + s]; r1[threadIdx.x] += r1[threadIdx.x + s]; }
        __syncthreads();
    }
    if (threadIdx.x == 0) { part[2 * blockIdx.x] = r0[0]; part[2 * blockIdx.x + 1] = r1[0]; }
}

// Validity of a prediction (phi, T, ux, uy planes of n sites): out[0] = 1 if
// any value is not finite, out[1] = bits of max(|ux|, |uy|) (non-negative
// floats order like their bit patterns).
__global__ void k_pred_check(const float* __restrict__ y, int64_t n, unsigned* out)
{
    unsigned bad = 0, umax = 0;
    for (int64_t k = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; k < 4 * n; k += (int64_t)gridDim.x * blockDim.x) {
        const float v = y[k];
        if (!isfinite(v)) bad = 1;
        else if (k >= 2 * n) umax = max(umax, __float_as_uint(fabsf(v)));
    }
    for (int o = 16; o > 0; o >>= 1) {
        bad |= __shfl_xor_sync(0xffffffffu, bad, o);
        umax = max(umax, __shfl_xor_sync(0xffffffffu, umax, o));
    }
    if ((threadIdx.x & 31) == 0) {
        if (bad) atomicOr(&out[0], 1u);
        atomicMax(&out[1], umax);
    }
}

int rel_l2(const float* a, const float* b, int64_t n, double* scratch, cudaStream_t s, double* out)
{
    const unsigned nb = blocks_for(n);
    k_l2_parts<<<nb, 256, 0, s>>>(a, b, n, scratch);
    std::vector<double> h(2 * nb);
    if (cudaMemcpyAsync(h.data(), scratch, sizeof(double) * 2 * nb, cudaMemcpyDeviceToHost, s) != cudaSuccess)
        return LF_ECUDA;
    int rc = wait_stream(s);
    if (rc != LF_OK) return rc;
    double s0 = 0, s1 = 0;
    for (unsigned i = 0; i < nb; ++i) { s0 += h[2 * i]; s1 += h[2 * i + 1]; }
    *out = s1 > 0 ? std::sqrt(s0 / s1) : std::sqrt(s0);
    return LF_OK;
}

}  // namespace

// Largest |u| (lattice units) a prediction may hand to the LB solver; the
// second-order equilibrium needs |u| well below the sound speed 1/sqrt(3).
constexpr float kMaxU = 0.2f;

extern "C" int lf_sur_run(lf_sur* s, lf_ctx* ctx, int K, int nwindows, int shadow_every, double threshold,
                          lf_sur_report* rep)
{
    lf::NvtxRange nvtx_range("lf_sur_run");
    if (!s || !ctx || !rep || K < 1 || nwindows < 0 || shadow_every < 1 || !(threshold > 0)) return LF_EINVAL;
    if (ctx->g.d != 2 || ctx->prec != LF_FP32 || !ctx->params.hydro || ctx->ens_member || ctx->g.nx != s->NX ||
        ctx->g.ny != s->NY)
        return LF_EINVAL;
    std::memset(rep, 0, sizeof(*rep));
    const int64_t N = (int64_t)s->NX * s->NY;
    const size_t fb = sizeof(float) * (size_t)N;
    // scratch: x, y (4 planes each), the plain phi of the shadow, populations, reduction partials
    unsigned char* buf = nullptr;
    const size_t bytes = 8 * fb + 9 * fb + fb + 8 * 2 * 152 * 8 + 1024;
    if (cudaMalloc((void**)&buf, bytes) != cudaSuccess) { cudaGetLastError(); return LF_ENOMEM; }
    float* x = (float*)buf;
    float* y = x + 4 * N;
    float* pop = y + 4 * N;
    float* phi_plain = pop + 9 * N;
    double* red = (double*)(phi_plain + N + 64);
    lf_params sp = ctx->params;
    sp.workspace = nullptr;
    sp.workspace_bytes = 0;
    sp.stream = ctx->stream;
    lf_ctx* shadow = nullptr;
    int rc = lf_create(&ctx->grid, &ctx->walls, &sp, &shadow);
    cudaEvent_t e0, e1;
    cudaEventCreate(&e0);
    cudaEventCreate(&e1);
    const cudaStream_t st = ctx->stream;
    // state copy between two contexts of the same shape, on the stream (no waits)
    auto copy_state = [&](lf_ctx* from, lf_ctx* to) {
        int r = fields_get_async(from, LF_FIELD_POP, pop, 9 * fb);
        if (r == LF_OK) r = fields_set_async(to, LF_FIELD_POP, pop, 9 * fb);
        if (r == LF_OK) r = fields_get_async(from, LF_FIELD_PHI, phi_plain, fb);
        if (r == LF_OK) r = fields_set_async(to, LF_FIELD_PHI, phi_plain, fb);
        if (r == LF_OK) r = fields_get_async(from, LF_FIELD_T, phi_plain, fb);
        if (r == LF_OK) r = fields_set_async(to, LF_FIELD_T, phi_plain, fb);
        return r;
    };
    for (int w = 0; w < nwindows && rc == LF_OK; ++w) {
        cudaEventRecord(e0, st);
        if (w % 2 == 1) {                                        // plain window
            rc = lf_step(ctx, K);
            if (rc == LF_OK) rc = wait_stream(st);
            cudaEventRecord(e1, st);
            cudaEventSynchronize(e1);
            float ms = 0;
            cudaEventElapsedTime(&ms, e0, e1);
            rep->t_plain_s += ms / 1e3;
            continue;
        }
        // surrogate window: x = (phi, T, ux, uy) of the current state
        const int which[4] = {LF_FIELD_PHI, LF_FIELD_T, LF_FIELD_UX, LF_FIELD_UY};
        for (int c = 0; c < 4 && rc == LF_OK; ++c) rc = fields_get_async(ctx, which[c], x + c * N, fb);
        if (rc == LF_OK) rc = lf_sur_predict(s, x, y, 1);
        unsigned chk[2] = {0u, 0u};
        if (rc == LF_OK) {
            unsigned* dchk = reinterpret_cast<unsigned*>(red);
            if (cudaMemsetAsync(dchk, 0, 2 * sizeof(unsigned), st) != cudaSuccess) rc = LF_ECUDA;
            if (rc == LF_OK) k_pred_check<<<152, 256, 0, st>>>(y, N, dchk);
            if (rc == LF_OK && cudaMemcpyAsync(chk, dchk, sizeof(chk), cudaMemcpyDeviceToHost, st) != cudaSuccess)
                rc = LF_ECUDA;
        }
        if (rc == LF_OK) rc = wait_stream(st);
        cudaEventRecord(e1, st);
        cudaEventSynchronize(e1);
        float ms_sur = 0;
        cudaEventElapsedTime(&ms_sur, e0, e1);
        rep->t_surrogate_s += ms_sur / 1e3;
        float umax;
        std::memcpy(&umax, &chk[1], sizeof(umax));
        if (rc == LF_OK && (chk[0] != 0u || !(umax <= kMaxU))) {   // not a usable state: take the plain window
            rep->rejected += 1;
            cudaEventRecord(e0, st);
            rc = lf_step(ctx, K);
            if (rc == LF_OK) rc = wait_stream(st);
            cudaEventRecord(e1, st);
            cudaEventSynchronize(e1);
            float ms = 0;
            cudaEventElapsedTime(&ms, e0, e1);
            rep->t_plain_s += ms / 1e3;
            rep->windows_done = w + 1;
            continue;
        }
        bool accept = true;
        if (rc == LF_OK && (w / 2) % shadow_every == 0) {        // plain shadow window as the check
            cudaEventRecord(e0, st);
            rc = copy_state(ctx, shadow);
            if (rc == LF_OK) rc = lf_step(shadow, K);
            lf_diag_t dp{}, ds{};
            if (rc == LF_OK) rc = lf_diag(shadow, &dp);
            if (rc == LF_OK) rc = lf_fields(shadow, LF_FIELD_PHI, phi_plain, fb, 1);
            double err_l2 = 0;
            if (rc == LF_OK) rc = rel_l2(y, phi_plain, N, red, st, &err_l2);
            if (rc == LF_OK) rc = lf_fields_set(shadow, LF_FIELD_PHI, y, fb, 1);
            if (rc == LF_OK) rc = lf_diag(shadow, &ds);
            if (rc == LF_ENONFINITE) rc = LF_OK, ds.k_peak = ds.s_peak = NAN;
            if (rc == LF_OK) rc = lf_fields_set(shadow, LF_FIELD_PHI, phi_plain, fb, 1);
            const double ek = dp.k_peak > 0 ? std::fabs(ds.k_peak / dp.k_peak - 1.0) : 0.0;
            const double es = dp.s_peak > 0 ? std::fabs(ds.s_peak / dp.s_peak - 1.0) : 0.0;
            double err = std::max(err_l2, std::max(ek, es));
            if (!std::isfinite(err)) err = 1e30;
            rep->shadow_checks += 1;
            rep->max_phi_l2_err = std::max(rep->max_phi_l2_err, err_l2);
            rep->max_sk_err = std::max(rep->max_sk_err, std::max(ek, es));
            rep->last_err = err;
            if (err > threshold) {
                accept = false;
                rep->fallbacks += 1;
                if (rc == LF_OK) rc = copy_state(shadow, ctx);
            }
            cudaEventRecord(e1, st);
            cudaEventSynchronize(e1);
            float ms = 0;
            cudaEventElapsedTime(&ms, e0, e1);
            rep->t_shadow_s += ms / 1e3;
        }
        if (rc == LF_OK && accept) {                             // hand the prediction to the solver
            rc = lf_fields_set(ctx, LF_FIELD_PHI, y, fb, 1);
            if (rc == LF_OK) rc = lf_fields_set(ctx, LF_FIELD_T, y + N, fb, 1);
            if (rc == LF_OK) {
                k_shift_u2d<<<blocks_for(N), 256, 0, st>>>(ctx->g, (float)ctx->params.n0, x + 2 * N, x + 3 * N,
                                                          y + 2 * N, y + 3 * N, (float*)ctx->f[ctx->fcur]);
                rc = cudaGetLastError() == cudaSuccess ? wait_stream(st) : LF_ECUDA;
            }
            rep->surrogate_windows += 1;
        }
        ctx->step += K;
        ctx->aux_valid = false;
        rep->windows_done = w + 1;
    }
    rep->windows_done = rc == LF_OK ? nwindows : rep->windows_done;
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    if (shadow) lf_destroy(shadow);
    cudaFree(buf);
    return rc;
}
