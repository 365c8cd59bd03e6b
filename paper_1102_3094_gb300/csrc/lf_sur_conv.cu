// lf_sur_conv.cu -- 3x3 convolution of NHWC BF16 activations on the 5th-gen
// tensor cores (tcgen05.mma, FP32 accumulator in tensor memory).
//
// Implicit GEMM: an output tile is 128 consecutive pixels of one image row
// (M = 128) times all COUT output channels (N), accumulated over the 9 taps x
// CIN input channels (K = 9 CIN, in steps of 16).  Activations live in a
// padded layout [B][NY + 2][NX + 2][C] whose one-pixel halo holds the
// boundary rule of the lattice (x periodic: the halo columns copy the
// opposite edge; y walls: the halo rows are zero).
//
// A persistent CTA owns a 128-pixel column block and a run of image rows and
// marches down them.  Input rows (130 pixels with the halo) sit in a 5-slot
// shared-memory ring in a pixel-major core-matrix layout ([k core][pixel][8
// channels], 16 bytes per pixel and core): the 8 pixels of a core matrix are
// contiguous, so the A operand of tap (dy, dx) is the ring row of dy with its
// descriptor start moved by dx pixels -- all 9 taps read the same three rows,
// which are loaded once.  The rows two ahead are prefetched with cp.async.
// The 9 weight taps stay in shared memory (K-major).  One thread issues the
// MMAs of row y into one of two TMEM accumulators while the warps run the
// epilogue of row y - 1 from the other.  With 64 output channels the CTA has
// 512 threads: a warp reads the TMEM lanes of its quarter (warp mod 4, 32
// pixels) and a quarter of the channels (warp / 4), so sixteen warps share
// the epilogue's memory latency (132 us against 157 us with four warps for
// 64 -> 64 at 8 x 256^2); the 16-channel last layer keeps 128 threads.
#include <cuda_bf16.h>

#include "lf_internal.cuh"
#include "lf_sur.h"
#include "lf_tc.cuh"

namespace lf {
namespace sur {

struct ConvArgs {
    const __nv_bfloat16* in;     // padded NHWC, CIN channels
    const __nv_bfloat16* w;      // [9][COUT][CIN], tap t = 3 (dy + 1) + (dx + 1)
    const float* bias;           // [COUT] or null
    const __nv_bfloat16* resid;  // padded NHWC COUT, added after the activation, or null
    const __nv_bfloat16* mask;   // padded NHWC COUT: out2 = out * (mask > 0), or null
    __nv_bfloat16* out;          // padded NHWC COUT, or null
    __nv_bfloat16* out2;         // padded NHWC COUT (masked copy of out), or null
    __nv_bfloat16* zout;         // padded NHWC COUT: pre-activation value, or null
    const float* x4;             // [B][NY][NX][4]: y4 = x4 + (acc + bias)[0..3], or null
    float* y4;
    int relu;
    int B, NY, NX;
    int* err;
};

template <int CIN, int COUT>
struct ConvSmem {
    static constexpr int RP = 130;                   // ring row: pixels x0 - 1 .. x0 + 128
    static constexpr int KC = CIN / 8;               // 16-byte channel groups (k cores)
    static constexpr int LBO_A = RP * 16;            // next k core of the A operand
    static constexpr int ROW_BYTES = KC * LBO_A;
    static constexpr int NSLOT = 5;                  // rows y - 1 .. y + 3
    static constexpr int B_TAP = COUT * CIN * 2;
    static constexpr int B_OFF = 0;
    static constexpr int R_OFF = 9 * B_TAP;
    static constexpr int BAR_OFF = R_OFF + NSLOT * ROW_BYTES;
    static constexpr int BYTES = BAR_OFF + 64;
    static constexpr int TMEM_COLS = 2 * COUT < 32 ? 32 : 2 * COUT;   // two accumulators
};

template <int COUT>
constexpr int conv_threads() { return COUT >= 64 ? 512 : 128; }

__device__ __forceinline__ int64_t pix_off(int b, int y, int x, int NY, int NX)
{
    return ((int64_t)b * (NY + 2) + (y + 1)) * (NX + 2) + (x + 1);   // padded pixel index
}

template <int CIN, int COUT>
__global__ void __launch_bounds__(conv_threads<COUT>(), 1) k_conv3x3(ConvArgs a, int rows_per_item)
{
    using S = ConvSmem<CIN, COUT>;
    constexpr int NT = conv_threads<COUT>();
    constexpr int PARTS = (NT / 128) < (COUT / 16) ? (NT / 128) : (COUT / 16);   // channel parts of the epilogue
    constexpr int CPP = COUT / PARTS;                                            // channels per part
    static_assert(CIN % 16 == 0 && COUT % 16 == 0 && COUT >= 16 && COUT <= 128, "MMA shape");
    extern __shared__ __align__(1024) unsigned char smem[];
    unsigned char* sB = smem + S::B_OFF;
    unsigned char* sR = smem + S::R_OFF;
    uint64_t* bar = reinterpret_cast<uint64_t*>(smem + S::BAR_OFF);
    uint32_t* tslot = reinterpret_cast<uint32_t*>(smem + S::BAR_OFF + 16);
    const int tid = threadIdx.x, warp = tid >> 5;
    const int NY = a.NY, NX = a.NX;
    const int ncb = NX / 128;
    const int nch = (NY + rows_per_item - 1) / rows_per_item;
    const int nitems = a.B * ncb * nch;
    constexpr uint32_t idesc = tc::idesc_bf16_f32(128, COUT);
    constexpr uint32_t SBO_B = (CIN / 8) * 128;

    if (warp == 0) tc::tmem_alloc(tslot, S::TMEM_COLS);
    if (tid == 0) {
        tc::mbar_init(&bar[0], 1);
        tc::mbar_init(&bar[1], 1);
        tc::fence_mbar_init();
    }
    // all 9 weight taps into shared memory (K-major core-matrix layout)
    for (int q = tid; q < 9 * COUT * (CIN / 8); q += NT) {
        const int t = q / (COUT * (CIN / 8)), rem = q - t * (COUT * (CIN / 8));
        const int n = rem / (CIN / 8), j = rem - n * (CIN / 8);
        tc::cp_async16(sB + t * S::B_TAP + tc::kmajor_offset(n, 8 * j, CIN), a.w + ((int64_t)t * COUT + n) * CIN + 8 * j);
    }
    tc::cp_async_commit_wait_all();
    tc::fence_proxy_async();
    tc::fence_before_sync();
    __syncthreads();
    tc::fence_after_sync();
    const uint32_t tmem = *tslot;
    const uint32_t lane_base = (uint32_t)((warp & 3) * 32) << 16;   // the warp's TMEM lane quarter
    const int part = warp >> 2;                                       // its share of the channels
    const int pix = tid & 127;                                        // pixel of the tile = TMEM lane
    uint32_t ph[2] = {0u, 0u};
    bool ok = true;

    // padded row pr (image row pr - 1) of image b, pixels x0 - 1 .. x0 + 128,
    // into ring slot pr mod 5; one 16-byte channel group per copy
    auto load_row = [&](int b, int pr, int x0) {
        unsigned char* dst = sR + (pr % S::NSLOT) * S::ROW_BYTES;
        const __nv_bfloat16* src = a.in + (((int64_t)b * (NY + 2) + pr) * (NX + 2) + x0) * CIN;
        for (int q = tid; q < S::RP * S::KC; q += NT) {
            const int px = q / S::KC, j = q - px * S::KC;
            tc::cp_async16(dst + j * S::LBO_A + px * 16, src + (int64_t)px * CIN + 8 * j);
        }
    };
    auto commit = [] { asm volatile("cp.async.commit_group;\n" ::: "memory"); };

    // MMAs of output row y: taps (dy, dx) read padded rows y + dy + 1 at pixel shift dx
    auto issue_row = [&](int y, uint32_t dcol) {
        const uint32_t ring = tc::smem_u32(sR), bbase = tc::smem_u32(sB);
#pragma unroll
        for (int t = 0; t < 9; ++t) {
            const int dy = t / 3 - 1, dx = t % 3 - 1;
            const uint32_t abase = ring + (uint32_t)(((y + dy + 1) % S::NSLOT) * S::ROW_BYTES + (dx + 1) * 16);
#pragma unroll
            for (int s = 0; s < CIN / 16; ++s)
                tc::mma_bf16(tmem + dcol, tc::smem_desc(abase + 2 * s * S::LBO_A, S::LBO_A, 128),
                             tc::smem_desc(bbase + t * S::B_TAP + 256 * s, 128, SBO_B), idesc,
                             (t > 0 || s > 0) ? 1u : 0u);
        }
    };

    // the thread's 16 channels of the bias, for the whole launch
    static_assert(CPP == 16, "one 16-channel group per thread in the epilogue");
    float bz[16];
#pragma unroll
    for (int i = 0; i < 16; ++i) bz[i] = (a.bias && part < PARTS) ? a.bias[part * CPP + i] : 0.f;
    // residual and mask inputs of the thread's pixel in row y, loaded before the
    // wait for the row's MMAs so that their latency overlaps it
    auto preload = [&](int b, int y, int x0, uint4* rp, uint4* mp) {
        if (part >= PARTS) return;
        const int64_t po = pix_off(b, y, x0 + pix, NY, NX);
        if (a.resid) {
            const uint4* rs = reinterpret_cast<const uint4*>(a.resid + po * COUT + part * CPP);
            rp[0] = rs[0];
            rp[1] = rs[1];
        }
        if (a.mask) {
            const uint4* ms = reinterpret_cast<const uint4*>(a.mask + po * COUT + part * CPP);
            mp[0] = ms[0];
            mp[1] = ms[1];
        }
    };

    // epilogue of output row y (TMEM accumulator at column dcol): thread = pixel
    auto epilogue = [&](int b, int y, int x0, uint32_t dcol, const uint4* rp, const uint4* mp) {
        if (part >= PARTS) return;
        const int x = x0 + pix;
        const int64_t po = pix_off(b, y, x, NY, NX);
        const bool halo_hi = (x == 0), halo_lo = (x == NX - 1);   // copies into columns NX + 1 / 0
        const int64_t po_h = halo_hi ? pix_off(b, y, NX, NY, NX) : pix_off(b, y, -1, NY, NX);
        {
            const int c0 = part * CPP;
            float v[16];
            tc::tmem_ld16(tmem + lane_base + dcol + (uint32_t)c0, v);
#pragma unroll
            for (int i = 0; i < 16; ++i) v[i] += bz[i];
            if (a.y4 && c0 == 0) {
                const int64_t q = (((int64_t)b * NY + y) * NX + x) * 4;
#pragma unroll
                for (int i = 0; i < 4; ++i) a.y4[q + i] = a.x4[q + i] + v[i];
            }
            __align__(16) __nv_bfloat16 hz[16], ho[16], hm[16];
            if (a.zout)
#pragma unroll
                for (int i = 0; i < 16; ++i) hz[i] = __float2bfloat16_rn(v[i]);
            if (a.relu)
#pragma unroll
                for (int i = 0; i < 16; ++i) v[i] = fmaxf(v[i], 0.f);
            if (a.resid) {
                __align__(16) __nv_bfloat16 r[16];
                reinterpret_cast<uint4*>(r)[0] = rp[0];
                reinterpret_cast<uint4*>(r)[1] = rp[1];
#pragma unroll
                for (int i = 0; i < 16; ++i) v[i] += __bfloat162float(r[i]);
            }
#pragma unroll
            for (int i = 0; i < 16; ++i) ho[i] = __float2bfloat16_rn(v[i]);
            if (a.mask) {
                __align__(16) __nv_bfloat16 m[16];
                reinterpret_cast<uint4*>(m)[0] = mp[0];
                reinterpret_cast<uint4*>(m)[1] = mp[1];
#pragma unroll
                for (int i = 0; i < 16; ++i) hm[i] = __bfloat162float(m[i]) > 0.f ? ho[i] : __float2bfloat16_rn(0.f);
            }
            auto store = [&](__nv_bfloat16* base, const __nv_bfloat16* h) {
                if (!base) return;
                const uint4* hv = reinterpret_cast<const uint4*>(h);
                uint4* d = reinterpret_cast<uint4*>(base + po * COUT + c0);
                d[0] = hv[0];
                d[1] = hv[1];
                if (halo_hi || halo_lo) {
                    uint4* dh = reinterpret_cast<uint4*>(base + po_h * COUT + c0);
                    dh[0] = hv[0];
                    dh[1] = hv[1];
                }
            };
            store(a.zout, hz);
            store(a.out, ho);
            if (a.mask) store(a.out2, hm);
        }
    };

    for (int item = blockIdx.x; item < nitems && ok; item += gridDim.x) {
        const int ch = item % nch, rest = item / nch;
        const int cb = rest % ncb, b = rest / ncb;
        const int x0 = cb * 128;
        const int ya = ch * rows_per_item, yb = min(ya + rows_per_item, NY);
        // prologue: padded rows ya .. ya + 2 (image rows ya - 1 .. ya + 1), then ya + 3
        load_row(b, ya, x0);
        load_row(b, ya + 1, x0);
        load_row(b, ya + 2, x0);
        commit();
        if (ya + 3 <= yb + 1) load_row(b, ya + 3, x0);
        commit();
        for (int y = ya; y < yb; ++y) {
            const uint32_t dcur = (uint32_t)((y & 1) * COUT), dprev = (uint32_t)(((y - 1) & 1) * COUT);
            // padded rows y .. y + 2 have landed; the epilogue of row y - 2 has
            // read accumulator y & 1
            asm volatile("cp.async.wait_group 1;\n" ::: "memory");
            tc::fence_proxy_async();
            tc::fence_before_sync();
            __syncthreads();
            tc::fence_after_sync();
            if (tid == 0) {
                issue_row(y, dcur);
                tc::mma_commit(&bar[y & 1]);
            }
            uint4 rp[2] = {}, mp[2] = {};
            if (y > ya) preload(b, y - 1, x0, rp, mp);
            if (y > ya) {   // MMAs of row y - 1 done: its ring slot and accumulator are free to use
                const bool w = tc::mbar_wait(&bar[(y - 1) & 1], ph[(y - 1) & 1]);
                ph[(y - 1) & 1] ^= 1;
                if (__syncthreads_or(!w)) { ok = false; break; }
                tc::fence_after_sync();
            }
            // prefetch padded row y + 4 into the slot of padded row y - 1
            if (y + 4 <= yb + 1) load_row(b, y + 4, x0);
            commit();
            if (y > ya) epilogue(b, y - 1, x0, dprev, rp, mp);
        }
        if (!ok) break;
        {   // last row of the item
            const int y = yb - 1;
            uint4 rp[2] = {}, mp[2] = {};
            preload(b, y, x0, rp, mp);
            const bool w = tc::mbar_wait(&bar[y & 1], ph[y & 1]);
            ph[y & 1] ^= 1;
            if (__syncthreads_or(!w)) { ok = false; break; }
            tc::fence_after_sync();
            epilogue(b, y, x0, (uint32_t)((y & 1) * COUT), rp, mp);
        }
        asm volatile("cp.async.wait_group 0;\n" ::: "memory");
        tc::fence_before_sync();
        __syncthreads();   // accumulators read and ring idle before the next item
        tc::fence_after_sync();
    }
    asm volatile("cp.async.wait_group 0;\n" ::: "memory");
    if (!ok && tid == 0) atomicExch(a.err, 1);
    tc::fence_before_sync();
    __syncthreads();
    if (warp == 0) tc::tmem_dealloc(tmem, S::TMEM_COLS);
}

template <int CIN, int COUT>
cudaError_t launch_conv(const ConvArgs& a, cudaStream_t s)
{
    using S = ConvSmem<CIN, COUT>;
    static unsigned long long attr_done = 0;      // per instantiation and device
    if (cudaError_t e = raise_smem_limit(k_conv3x3<CIN, COUT>, (int)S::BYTES, &attr_done); e != cudaSuccess) return e;
    // rows per item: at least ~4 rows (prologue of 4 loaded rows) and about
    // two items per SM over the whole launch
    const int cols = a.B * (a.NX / 128);
    int rpi = (int)(((int64_t)cols * a.NY + 2 * 152 - 1) / (2 * 152));
    if (rpi < 4) rpi = 4;
    if (rpi > a.NY) rpi = a.NY;
    const int nitems = cols * ((a.NY + rpi - 1) / rpi);
    const int blocks = nitems < 152 ? nitems : 152;
    k_conv3x3<CIN, COUT><<<blocks, conv_threads<COUT>(), S::BYTES, s>>>(a, rpi);
    return cudaGetLastError();
}

cudaError_t conv3x3(int cin, int cout, const ConvArgs& a, cudaStream_t s)
{
    if (cin == 16 && cout == 64) return launch_conv<16, 64>(a, s);
    if (cin == 64 && cout == 64) return launch_conv<64, 64>(a, s);
    if (cin == 64 && cout == 16) return launch_conv<64, 16>(a, s);
    return cudaErrorInvalidValue;
}

// ---------------------------------------------------------------------------
// Weight gradient of a 3x3 convolution on the tensor cores:
//   dW[t][o][i] = sum_p h[p + off_t][i] g[p][o]
// For each tap a GEMM D_t = A B^T with K = pixels, M = 64 (the 64-channel
// side: i for CIN = 64, else o) and N = the other side.  Both operands are
// read MN-major straight from rows staged in the pixel-major core-matrix
// layout of the forward kernel ([channel group][pixel][8 channels]): a core
// matrix is 8 consecutive pixels (K) of 8 channels (MN), so the tap shift dx
// is a 16-byte move of the descriptor start and nothing is transposed.  A
// work item is a run of row tiles (128 pixels of one image row) for one
// group of taps; it accumulates all of its rows in TMEM (one M = 64
// accumulator per tap) and writes one FP32 partial, summed by
// k_wgrad_reduce.  For 64 -> 64 the taps are split in three groups by dy
// (TMEM holds 3 x 64 columns); otherwise one group holds all nine.
// ---------------------------------------------------------------------------
// threads of the weight-gradient kernel (its time goes to the chain of
// M = 64 MMAs of each row, not to the staging copies: 256 threads measured
// the same, 214 us against 208 us for 64 -> 64 at 8 x 256^2)
constexpr int kWgThreads = 128;

template <int CIN, int COUT>
struct WgCfg {
    static constexpr bool HA = CIN == 64;                  // h is the M = 64 operand
    static constexpr int NB = HA ? COUT : CIN;             // N of the GEMM
    static constexpr int NG = (CIN == 64 && COUT == 64) ? 3 : 1;
    static constexpr int TG = 9 / NG;                      // taps per group
    static constexpr int SLICES = (2 * 152) / NG;          // items per group
    static constexpr int RH = 130, RG = 128;               // pixels per staged h / g row
    static constexpr int HROW = (CIN / 8) * RH * 16, GROW = (COUT / 8) * RG * 16;
    static constexpr int NSH = NG == 3 ? 4 : 6, NSG = 4;
    static constexpr int H_OFF = 0, G_OFF = NSH * HROW, BAR_OFF = G_OFF + NSG * GROW;
    static constexpr int BYTES = BAR_OFF + 64;
    static constexpr int TCOLS = TG * NB <= 32 ? 32 : (TG * NB <= 64 ? 64 : (TG * NB <= 128 ? 128 : 256));
    static constexpr size_t PART = (size_t)NG * SLICES * TG * 64 * NB;   // floats
};

struct WgArgs {
    const __nv_bfloat16* h;      // padded NHWC CIN
    const __nv_bfloat16* g;      // padded NHWC COUT
    float* part;                 // [NG][SLICES][TG][64][NB]
    int B, NY, NX;
    int* err;
};

template <int CIN, int COUT>
__global__ void __launch_bounds__(kWgThreads, 1) k_conv_wgrad(WgArgs a)
{
    using S = WgCfg<CIN, COUT>;
    extern __shared__ __align__(1024) unsigned char smem[];
    unsigned char* sH = smem + S::H_OFF;
    unsigned char* sG = smem + S::G_OFF;
    uint64_t* bar = reinterpret_cast<uint64_t*>(smem + S::BAR_OFF);      // one per g slot
    uint32_t* tslot = reinterpret_cast<uint32_t*>(smem + S::BAR_OFF + 48);
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    const int NY = a.NY, NX = a.NX;
    const int ncb = NX / 128;
    const int64_t R = (int64_t)a.B * ncb * NY;                 // row tiles, ordered (b, cb, y)
    constexpr uint32_t idesc = tc::idesc_bf16_f32(64, S::NB) | (1u << 15) | (1u << 16);   // both MN-major

    if (warp == 0) tc::tmem_alloc(tslot, S::TCOLS);
    if (tid == 0) {
        for (int k = 0; k < S::NSG; ++k) tc::mbar_init(&bar[k], 1);
        tc::fence_mbar_init();
    }
    tc::fence_before_sync();
    __syncthreads();
    tc::fence_after_sync();
    const uint32_t tmem = *tslot;
    uint32_t ph[S::NSG] = {};
    bool ok = true;

    auto commit = [] { asm volatile("cp.async.commit_group;\n" ::: "memory"); };
    // padded h row pr, pixels x0 - 1 .. x0 + 128, into h slot pr mod NSH
    auto load_h = [&](int b, int pr, int x0) {
        unsigned char* dst = sH + (pr % S::NSH) * S::HROW;
        const __nv_bfloat16* src = a.h + (((int64_t)b * (NY + 2) + pr) * (NX + 2) + x0) * CIN;
        for (int q = tid; q < S::RH * (CIN / 8); q += kWgThreads) {
            const int px = q / (CIN / 8), j = q - px * (CIN / 8);
            tc::cp_async16(dst + j * (S::RH * 16) + px * 16, src + (int64_t)px * CIN + 8 * j);
        }
    };
    // g row y, pixels x0 .. x0 + 127, into g slot y mod NSG
    auto load_g = [&](int b, int y, int x0) {
        unsigned char* dst = sG + (y % S::NSG) * S::GROW;
        const __nv_bfloat16* src = a.g + (((int64_t)b * (NY + 2) + y + 1) * (NX + 2) + x0 + 1) * COUT;
        for (int q = tid; q < S::RG * (COUT / 8); q += kWgThreads) {
            const int px = q / (COUT / 8), j = q - px * (COUT / 8);
            tc::cp_async16(dst + j * (S::RG * 16) + px * 16, src + (int64_t)px * COUT + 8 * j);
        }
    };
    // everything output row y of this group reads that is not already staged
    // by earlier rows: g row y and the newest h row(s)
    auto load_rows_for = [&](int b, int y, int x0, int gi, bool first) {
        load_g(b, y, x0);
        if (S::NG == 3) {
            load_h(b, y + gi, x0);                 // padded row y + dy + 1, dy = gi - 1
        } else if (first) {
            load_h(b, y, x0); load_h(b, y + 1, x0); load_h(b, y + 2, x0);
        } else {
            load_h(b, y + 2, x0);
        }
    };

    for (int item = blockIdx.x; item < S::NG * S::SLICES && ok; item += gridDim.x) {
        const int gi = item / S::SLICES, sl = item - gi * S::SLICES;
        const int64_t r0 = R * sl / S::SLICES, r1 = R * (sl + 1) / S::SLICES;
        const int t0 = gi * S::TG;
        bool first_row = true;
        for (int64_t r = r0; r < r1 && ok;) {
            // one run of consecutive rows of one (image, column block)
            const int64_t bc = r / NY;
            const int ya = (int)(r - bc * NY);
            const int64_t rend = min(r1, (bc + 1) * NY);
            const int yb = ya + (int)(rend - r);
            const int cb = (int)(bc % ncb), b = (int)(bc / ncb);
            const int x0 = cb * 128;
            load_rows_for(b, ya, x0, gi, true);
            commit();
            if (ya + 1 < yb) load_rows_for(b, ya + 1, x0, gi, false);
            commit();
            for (int y = ya; y < yb; ++y) {
                asm volatile("cp.async.wait_group 1;\n" ::: "memory");   // rows of output row y landed
                tc::fence_proxy_async();
                tc::fence_before_sync();
                __syncthreads();
                tc::fence_after_sync();
                if (tid == 0) {
                    const uint32_t gb = tc::smem_u32(sG + (y % S::NSG) * S::GROW);
#pragma unroll
                    for (int j = 0; j < S::TG; ++j) {
                        const int t = t0 + j, dy = t / 3 - 1, dx = t % 3 - 1;
                        const uint32_t hb = tc::smem_u32(sH + ((y + dy + 1) % S::NSH) * S::HROW) + (dx + 1) * 16;
#pragma unroll
                        for (int s = 0; s < 8; ++s) {            // 16 pixels per MMA
                            const uint64_t hd = tc::smem_desc(hb + 256 * s, 128, S::RH * 16);
                            const uint64_t gd = tc::smem_desc(gb + 256 * s, 128, S::RG * 16);
                            tc::mma_bf16(tmem + (uint32_t)(j * S::NB), S::HA ? hd : gd, S::HA ? gd : hd, idesc,
                                         (first_row && s == 0) ? 0u : 1u);
                        }
                    }
                    tc::mma_commit(&bar[y % S::NSG]);
                }
                first_row = false;
                if (y >= ya + 2) {   // MMAs of row y - 2 done: its slots may be refilled
                    const int k = (y - 2) % S::NSG;
                    const bool w = tc::mbar_wait(&bar[k], ph[k]);
                    ph[k] ^= 1;
                    if (__syncthreads_or(!w)) { ok = false; break; }
                }
                if (y + 2 < yb) load_rows_for(b, y + 2, x0, gi, false);
                commit();
            }
            if (!ok) break;
            for (int y = max(ya, yb - 2); y < yb; ++y) {   // the last two rows' MMAs
                const int k = y % S::NSG;
                const bool w = tc::mbar_wait(&bar[k], ph[k]);
                ph[k] ^= 1;
                if (__syncthreads_or(!w)) { ok = false; break; }
            }
            asm volatile("cp.async.wait_group 0;\n" ::: "memory");
            tc::fence_before_sync();
            __syncthreads();
            tc::fence_after_sync();
            r = rend;
        }
        if (!ok) break;
        // partial of this item: M = 64 accumulator rows 16 w + l sit in lanes 32 w + l, l < 16
        // (warps 0..3, one TMEM lane quarter each)
        float* dst = a.part + ((size_t)item * S::TG) * 64 * S::NB;
        const int m = 16 * warp + lane;
#pragma unroll
        for (int j = 0; j < (warp < 4 ? S::TG : 0); ++j)
#pragma unroll
            for (int c0 = 0; c0 < S::NB; c0 += 16) {
                float v[16];
                tc::tmem_ld16(tmem + ((uint32_t)(warp * 32) << 16) + (uint32_t)(j * S::NB + c0), v);
                if (lane < 16)
#pragma unroll
                    for (int i = 0; i < 16; ++i) dst[((size_t)j * 64 + m) * S::NB + c0 + i] = first_row ? 0.f : v[i];
            }
        tc::fence_before_sync();
        __syncthreads();   // accumulators read before the next item's first MMA
        tc::fence_after_sync();
    }
    asm volatile("cp.async.wait_group 0;\n" ::: "memory");
    if (!ok && tid == 0) atomicExch(a.err, 1);
    tc::fence_before_sync();
    __syncthreads();
    if (warp == 0) tc::tmem_dealloc(tmem, S::TCOLS);
}

// dW[t][o][i] = sum over the group's items of part[item][t - t0][m][n]
template <int CIN, int COUT>
__global__ void k_wgrad_reduce(const float* __restrict__ part, float* __restrict__ dW)
{
    using S = WgCfg<CIN, COUT>;
    const int idx = blockIdx.x * blockDim.x + threadIdx.x;
    if (idx >= 9 * COUT * CIN) return;
    const int t = idx / (COUT * CIN), rem = idx - t * COUT * CIN;
    const int o = rem / CIN, i = rem - o * CIN;
    const int gi = t / S::TG, j = t - gi * S::TG;
    const int m = S::HA ? i : o, n = S::HA ? o : i;
    float acc = 0.f;
    for (int sl = 0; sl < S::SLICES; ++sl)
        acc += part[((((size_t)gi * S::SLICES + sl) * S::TG + j) * 64 + m) * S::NB + n];
    dW[idx] = acc;
}

template <int CIN, int COUT>
cudaError_t launch_wgrad(const __nv_bfloat16* h, const __nv_bfloat16* g, int B, int NY, int NX, float* part,
                         size_t part_floats, float* dW, int* err, cudaStream_t s)
{
    using S = WgCfg<CIN, COUT>;
    static unsigned long long attr_done = 0;      // per instantiation and device
    if (cudaError_t e = raise_smem_limit(k_conv_wgrad<CIN, COUT>, (int)S::BYTES, &attr_done); e != cudaSuccess)
        return e;
    if (part_floats < S::PART) return cudaErrorInvalidValue;
    WgArgs a{h, g, part, B, NY, NX, err};
    k_conv_wgrad<CIN, COUT><<<152, kWgThreads, S::BYTES, s>>>(a);
    const int n = 9 * COUT * CIN;
    k_wgrad_reduce<CIN, COUT><<<(n + 255) / 256, 256, 0, s>>>(part, dW);
    return cudaGetLastError();
}

cudaError_t conv3x3_wgrad(int cin, int cout, const __nv_bfloat16* h, const __nv_bfloat16* g, int B, int NY, int NX,
                          float* part, size_t part_floats, float* dW, int* err, cudaStream_t s)
{
    if (cin == 16 && cout == 64) return launch_wgrad<16, 64>(h, g, B, NY, NX, part, part_floats, dW, err, s);
    if (cin == 64 && cout == 64) return launch_wgrad<64, 64>(h, g, B, NY, NX, part, part_floats, dW, err, s);
    if (cin == 64 && cout == 16) return launch_wgrad<64, 16>(h, g, B, NY, NX, part, part_floats, dW, err, s);
    return cudaErrorInvalidValue;
}

// scratch floats the weight-gradient partials need for a (cin, cout) layer
size_t wgrad_part_floats(int cin, int cout)
{
    if (cin == 16 && cout == 64) return WgCfg<16, 64>::PART;
    if (cin == 64 && cout == 64) return WgCfg<64, 64>::PART;
    if (cin == 64 && cout == 16) return WgCfg<64, 16>::PART;
    return 0;
}

}  // namespace sur
}  // namespace lf

extern "C" int lf_sur_conv3x3(int B, int NY, int NX, int cin, int cout, const void* in, const void* w,
                              const float* bias, int relu, const void* resid, const void* mask, void* out,
                              void* out2, void* zout, const float* x4, float* y4, int* err, void* stream)
{
    using namespace lf;
    if (B < 1 || NY < 1 || NX < 128 || NX % 128 != 0 || !in || !w || !err) return LF_EINVAL;
    if (!((cin == 16 && cout == 64) || (cin == 64 && cout == 64) || (cin == 64 && cout == 16))) return LF_EINVAL;
    if ((mask && !out2) || (!out && !zout && !y4) || (y4 && !x4)) return LF_EINVAL;
    if (((uintptr_t)in | (uintptr_t)w | (uintptr_t)out | (uintptr_t)out2 | (uintptr_t)zout | (uintptr_t)resid |
         (uintptr_t)mask) & 15)
        return LF_EINVAL;                                           // 16-byte vector accesses
    sur::ConvArgs a{};
    a.in = (const __nv_bfloat16*)in;
    a.w = (const __nv_bfloat16*)w;
    a.bias = bias;
    a.resid = (const __nv_bfloat16*)resid;
    a.mask = (const __nv_bfloat16*)mask;
    a.out = (__nv_bfloat16*)out;
    a.out2 = (__nv_bfloat16*)out2;
    a.zout = (__nv_bfloat16*)zout;
    a.x4 = x4;
    a.y4 = y4;
    a.relu = relu;
    a.B = B; a.NY = NY; a.NX = NX;
    a.err = err;
    return sur::conv3x3(cin, cout, a, (cudaStream_t)stream) == cudaSuccess ? LF_OK : LF_ECUDA;
}

extern "C" int lf_sur_conv3x3_wgrad(int B, int NY, int NX, int cin, int cout, const void* h, const void* g,
                                    float* part, size_t part_floats, float* dW, int* err, void* stream)
{
    using namespace lf;
    if (B < 1 || NY < 1 || NX < 128 || NX % 128 != 0 || !h || !g || !part || !dW || !err) return LF_EINVAL;
    if (!((cin == 16 && cout == 64) || (cin == 64 && cout == 64) || (cin == 64 && cout == 16))) return LF_EINVAL;
    if (((uintptr_t)h | (uintptr_t)g) & 15) return LF_EINVAL;
    if (part_floats < sur::wgrad_part_floats(cin, cout)) return LF_EINVAL;
    return sur::conv3x3_wgrad(cin, cout, (const __nv_bfloat16*)h, (const __nv_bfloat16*)g, B, NY, NX, part,
                              part_floats, dW, err, (cudaStream_t)stream) == cudaSuccess ? LF_OK : LF_ECUDA;
}

extern "C" size_t lf_sur_wgrad_scratch_floats(int cin, int cout) { return lf::sur::wgrad_part_floats(cin, cout); }
