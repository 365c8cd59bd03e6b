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
// One persistent CTA per SM takes an equal contiguous share of the output
// rows (ordered image, 128-pixel column block, row) and marches down them.
// Input rows (130 pixels with the halo) sit in an 8-slot shared-memory ring,
// K-major: with 64 channels each pixel is a 128-byte row of the 128-byte
// swizzled layout; with 16, the interleaved core-matrix layout ([k core]
// [pixel][8 channels]).  Either way the A operand of tap (dy, dx) is the ring
// row of dy with its descriptor start moved by dx pixels -- all 9 taps read
// the same three rows, which are loaded once.  The 9 weight taps stay in
// shared memory in the same K-major layouts.  A residual that is the layer's
// own input is read from the ring as well.  The warps have fixed roles that
// hand work over through mbarriers:
//   * a producer warp loads the weights and then each row by TMA as soon as
//     its ring slot is free (64 channels: one box of 130 pixels in the
//     128-byte swizzled layout; 16: one 8-channel box per k core);
//   * an MMA warp issues an input row's MMAs once it has landed and the
//     accumulator slot of the output row it starts has been read, and commits
//     the output row it completes and the input row it no longer needs;
//   * the epilogue warps (a TMEM lane quarter and 16 channels each: sixteen
//     warps for 64 output channels, four for 16) read an accumulator, release
//     it, and add bias, activation, residual and mask on the way out.
// Each input row feeds the three output rows it touches: the dy taps of one
// tap column dx are stacked along N (one MMA with N = 3 COUT per dx and K
// step), and output rows accumulate in eight TMEM slots of COUT columns
// (slot (-r) mod 8 for the CTA's r-th row, so the three rows are adjacent).
// So the loads of the rows ahead, the MMAs of the next rows and the epilogue
// of the current one overlap, with up to five rows between MMA and epilogue.
#include <cuda.h>
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
    // 64 input channels: a ring row is 130 pixel rows of 128 bytes in the
    // 128-byte swizzled K-major layout (16-byte chunk c of pixel p at chunk
    // c ^ (p mod 8)), one TMA box per row; fewer channels: core-matrix
    // interleaved rows ([k core][pixel][8 channels]), one box per k core
    static constexpr bool SW = CIN == 64;
    static constexpr int LBO_A = 2176;               // interleaved: next k core, 130 x 16 bytes padded to 128
    static constexpr int TX_BYTES = KC * RP * 16;    // bytes one row's TMA copies bring
    static constexpr int ROW_BYTES = SW ? 17 * 1024 : KC * LBO_A;
    static constexpr int NSLOT = 8;                  // ring of input rows
    static constexpr int NACC = 8;                   // TMEM accumulator slots of COUT columns (output rows)
    static constexpr int B_TAP = COUT * CIN * 2;
    static constexpr int B_OFF = 0;
    static constexpr int R_OFF = 9 * B_TAP;
    static constexpr int BAR_OFF = R_OFF + NSLOT * ROW_BYTES;
    static constexpr int NBAR = 2 * NSLOT + 2 * NACC + 2;   // full, empty, acc full, acc empty, done, weights
    static constexpr int BYTES = BAR_OFF + NBAR * 8 + 16;
    static constexpr int TMEM_COLS = NACC * COUT < 32 ? 32 : NACC * COUT;
    static_assert(R_OFF % 1024 == 0 && (!SW || ROW_BYTES % 1024 == 0) && LBO_A % 128 == 0 && LBO_A >= RP * 16,
                  "TMA destinations 1024-byte aligned (swizzle pattern) and 128-byte aligned");
    static_assert((TMEM_COLS & (TMEM_COLS - 1)) == 0 && TMEM_COLS <= 512, "TMEM allocation");
};

// warps: the epilogue warps (one TMEM lane quarter and 16 channels each),
// then one TMA producer warp and one MMA warp
template <int COUT>
constexpr int conv_epi_warps() { return COUT >= 64 ? 16 : 4; }
template <int COUT>
constexpr int conv_threads() { return 32 * (conv_epi_warps<COUT>() + 2); }

__device__ __forceinline__ int64_t pix_off(int b, int y, int x, int NY, int NX)
{
    return ((int64_t)b * (NY + 2) + (y + 1)) * (NX + 2) + (x + 1);   // padded pixel index
}

// The CTA's rows are a contiguous share [r0, r1) of all B * (NX / 128) * NY
// output rows, ordered (image, column block, row); a segment is a maximal run
// of them in one (image, column block).
struct ConvSeg {
    int b, x0, ya, yb;
};
__device__ __forceinline__ ConvSeg conv_segment(int64_t q, int64_t r1, int NY, int ncb)
{
    const int64_t col = q / NY;
    ConvSeg g;
    g.ya = (int)(q - col * NY);
    g.yb = (int)min((int64_t)NY, (int64_t)g.ya + (r1 - q));
    g.b = (int)(col / ncb);
    g.x0 = (int)(col - (int64_t)g.b * ncb) * 128;
    return g;
}

template <int CIN, int COUT>
__global__ void __launch_bounds__(conv_threads<COUT>(), 1)
    k_conv3x3(const __grid_constant__ CUtensorMap tin, const __grid_constant__ CUtensorMap tw, ConvArgs a)
{
    using S = ConvSmem<CIN, COUT>;
    constexpr int EW = conv_epi_warps<COUT>();
    constexpr int NT = conv_threads<COUT>();
    constexpr int PARTS = (EW / 4) < (COUT / 16) ? (EW / 4) : (COUT / 16);   // channel parts of the epilogue
    constexpr int CPP = COUT / PARTS;                                          // channels per part
    static_assert(CIN % 16 == 0 && COUT % 16 == 0 && COUT >= 16 && COUT <= 128, "MMA shape");
    static_assert(CPP == 16, "one 16-channel group per thread in the epilogue");
    extern __shared__ __align__(1024) unsigned char smem[];
    unsigned char* sB = smem + S::B_OFF;
    unsigned char* sR = smem + S::R_OFF;
    uint64_t* full = reinterpret_cast<uint64_t*>(smem + S::BAR_OFF);   // ring slot loaded
    uint64_t* empty = full + S::NSLOT;                                   // ring slot read (MMAs, ring residual)
    uint64_t* accf = empty + S::NSLOT;                                   // accumulator complete
    uint64_t* acce = accf + S::NACC;                                     // accumulator read by the epilogue
    uint64_t* done = acce + S::NACC;                                     // every MMA of the CTA complete
    uint64_t* wbar = done + 1;                                           // weights in shared memory
    uint32_t* tslot = reinterpret_cast<uint32_t*>(wbar + 1);
    volatile int* abort_flag = reinterpret_cast<volatile int*>(tslot + 1);
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    const int NY = a.NY, NX = a.NX, ncb = NX / 128;
    const int64_t R = (int64_t)a.B * ncb * NY;
    const int64_t r0 = R * blockIdx.x / gridDim.x, r1 = R * (blockIdx.x + 1) / gridDim.x;
    // a residual that is the layer's own input is read from the input ring (the
    // output row y's residual is padded row y + 1, pixels 1 .. 128 of its slot);
    // a slot is then free once its MMAs and that read are done
    const bool ring_res = CIN == COUT && a.resid != nullptr &&
                          (const void*)a.resid == (const void*)a.in;

    if (warp == 0) tc::tmem_alloc(tslot, S::TMEM_COLS);
    if (tid == 0) {
        for (int i = 0; i < S::NSLOT; ++i) {
            tc::mbar_init(&full[i], 1);
            tc::mbar_init(&empty[i], ring_res ? 1 + EW : 1);
        }
        for (int i = 0; i < S::NACC; ++i) {
            tc::mbar_init(&accf[i], 1);
            tc::mbar_init(&acce[i], EW);
        }
        tc::mbar_init(done, 1);
        tc::mbar_init(wbar, S::SW ? 1 : EW);
        // TMA destinations: 128-byte aligned, 1024 for the swizzle pattern
        *abort_flag = (tc::smem_u32(smem) & (S::SW ? 1023u : 127u)) ? 1 : 0;
        tc::fence_mbar_init();
    }
    tc::fence_before_sync();
    __syncthreads();
    tc::fence_after_sync();
    const uint32_t tmem = *tslot;
    const bool start = *abort_flag == 0;

    if (warp == EW) {
        // TMA producer: the weights, then padded rows ya .. yb + 1 of each
        // segment into the ring, one box per row (64 channels, swizzled) or per
        // k core (8 channels)
        if (lane == 0 && start) {
            if (S::SW) {   // the 9 weight taps, one swizzled box of COUT rows x 64 channels each
                tc::mbar_arrive_expect_tx(wbar, 9 * S::B_TAP);
                for (int t = 0; t < 9; ++t)
                    tc::tma_load_3d(sB + (3 * (t % 3) + t / 3) * S::B_TAP, &tw, 0, 0, t, wbar);
            }
            uint32_t ld = 0;
            bool ok = true;
            for (int64_t q = r0; q < r1 && ok;) {
                const ConvSeg g = conv_segment(q, r1, NY, ncb);
                for (int pr = g.ya; pr <= g.yb + 1; ++pr, ++ld) {
                    const uint32_t s = ld % S::NSLOT;
                    if (!tc::mbar_wait_or_abort(&empty[s], ((ld / S::NSLOT) & 1) ^ 1, abort_flag)) { ok = false; break; }
                    tc::mbar_arrive_expect_tx(&full[s], S::TX_BYTES);
                    if (S::SW)
                        tc::tma_load_3d(sR + s * S::ROW_BYTES, &tin, 0, g.x0, g.b * (NY + 2) + pr, &full[s]);
                    else
#pragma unroll
                        for (int j = 0; j < S::KC; ++j)
                            tc::tma_load_3d(sR + s * S::ROW_BYTES + j * S::LBO_A, &tin, 8 * j, g.x0,
                                            g.b * (NY + 2) + pr, &full[s]);
                }
                q += g.yb - g.ya;
            }
            // leave no copy in flight: the weights and the newest load of every
            // slot have landed (after an abort the MMA warp may not have waited)
            if (S::SW) tc::mbar_wait(wbar, 0);
            for (uint32_t k = ld > (uint32_t)S::NSLOT ? ld - S::NSLOT : 0u; k < ld; ++k)
                tc::mbar_wait(&full[k % S::NSLOT], (k / S::NSLOT) & 1);
        }
    } else if (warp == EW + 1) {
        // MMA issue, one input row at a time: padded row p of a segment feeds
        // output rows p, p - 1, p - 2 through taps dy = 0, 1, 2.  Output row r
        // (CTA count) accumulates in TMEM slot (-r) mod NACC, so the three rows
        // an input row feeds sit in consecutive slots and one MMA with
        // N = 3 COUT (the dy taps of one dx stacked) covers them; where the
        // slots wrap around the end of TMEM the MMA is split in two.
        if (lane == 0 && start) {
            constexpr uint32_t SBO_B = (CIN / 8) * 128;
            const uint32_t ring = tc::smem_u32(sR);
            const uint32_t bbase = tc::smem_u32(sB);
            const uint64_t bdesc0 = tc::smem_desc(bbase, 128, SBO_B);
            auto slot = [](uint32_t r) { return (0u - r) % (uint32_t)S::NACC; };
            uint32_t ld0 = 0, rs = 0;   // the segment's first load and first output row
            bool ok = tc::mbar_wait_or_abort(wbar, 0, abort_flag), issued = false;
            for (int64_t q = r0; q < r1 && ok;) {
                const ConvSeg g = conv_segment(q, r1, NY, ncb);
                const int n = g.yb - g.ya;
                for (int i = 0; i < n + 2; ++i) {   // padded row p = ya + i, load ld0 + i
                    const uint32_t k = ld0 + i;
                    const int dlo = i - (n - 1) > 0 ? i - (n - 1) : 0;   // taps whose output row is in the segment
                    const int dhi = i < 2 ? i : 2;
                    if (i < n)   // output row p starts: its slot must have been read
                        ok = tc::mbar_wait_or_abort(&acce[slot(rs + i)], (((rs + i) / S::NACC) & 1) ^ 1, abort_flag);
                    if (ok) ok = tc::mbar_wait_or_abort(&full[k % S::NSLOT], (k / S::NSLOT) & 1, abort_flag);
                    if (!ok) break;
                    tc::fence_after_sync();
                    // descriptors at the row's start (A) and at tap position 0 (B); an
                    // offset within shared memory adds (bytes >> 4) to the start-address
                    // field, so the (dx, s) offsets below are constants
                    const uint32_t abase = ring + (k % S::NSLOT) * S::ROW_BYTES;
                    const uint64_t a0 = S::SW ? tc::smem_desc_sw128(abase) : tc::smem_desc(abase, S::LBO_A, 128);
                    const uint64_t b0 = S::SW ? tc::smem_desc_sw128(bbase) : bdesc0;
                    // the taps dlo .. dhi go to slots slot(rs + i - dlo) onwards: one piece,
                    // or two where the slots wrap around the end of TMEM
                    const uint32_t c = slot(rs + i - dlo);
                    const int m = dhi - dlo + 1;
                    const int m1 = (int)c + m <= S::NACC ? m : S::NACC - (int)c, m2 = m - m1;
                    const uint32_t d1 = tmem + c * COUT, id1 = tc::idesc_bf16_f32(128, m1 * COUT);
                    const uint32_t id2 = tc::idesc_bf16_f32(128, (m2 > 0 ? m2 : 1) * COUT);
                    const uint64_t b1 = b0 + (uint64_t)((dlo * S::B_TAP) >> 4), b2 = b1 + (uint64_t)((m1 * S::B_TAP) >> 4);
                    constexpr int AS = S::SW ? 32 : 2 * S::LBO_A, AX = S::SW ? 128 : 16;   // A: K step, pixel
                    constexpr int BS = S::SW ? 32 : 256;                                   // B: K step
#pragma unroll
                    for (int dx = 0; dx < 3; ++dx)
#pragma unroll
                        for (int s = 0; s < CIN / 16; ++s) {
                            const uint64_t ad = a0 + (uint64_t)((dx * AX + s * AS) >> 4);
                            const uint64_t bo = (uint64_t)((3 * dx * S::B_TAP + s * BS) >> 4);
                            if (dx == 0 && s == 0 && dlo == 0) {
                                // the new accumulator of row p (tap dy = 0, slot c) starts from
                                // zero; the taps dy = 1 .. dhi of the other rows accumulate
                                tc::mma_bf16(d1, ad, b0, tc::idesc_bf16_f32(128, COUT), 0u);
                                if (dhi > 0) {
                                    const uint32_t c1 = (c + 1) % (uint32_t)S::NACC;
                                    const int n1 = (int)c1 + dhi <= S::NACC ? dhi : S::NACC - (int)c1;
                                    tc::mma_bf16(tmem + c1 * COUT, ad, b0 + (uint64_t)(S::B_TAP >> 4),
                                                 tc::idesc_bf16_f32(128, n1 * COUT), 1u);
                                    if (n1 < dhi)
                                        tc::mma_bf16(tmem, ad, b0 + (uint64_t)(((1 + n1) * S::B_TAP) >> 4),
                                                     tc::idesc_bf16_f32(128, (dhi - n1) * COUT), 1u);
                                }
                            } else {
                                tc::mma_bf16(d1, ad, b1 + bo, id1, 1u);
                                if (m2 > 0) tc::mma_bf16(tmem, ad, b2 + bo, id2, 1u);
                            }
                        }
                    issued = true;
                    tc::mma_commit(&empty[k % S::NSLOT]);                       // the row's last MMA
                    if (ring_res && (i == 0 || i == n + 1))   // no residual read of this row follows
                        tc::mbar_arrive_cnt(&empty[k % S::NSLOT], EW);
                    if (dhi == 2) tc::mma_commit(&accf[slot(rs + i - 2)]);      // output row p - 2 is complete
                }
                ld0 += n + 2;
                rs += n;
                q += n;
            }
            if (issued) {   // leave no MMA in flight
                tc::mma_commit(done);
                tc::mbar_wait(done, 0);
            }
        }
    } else if (start) {
        // the 9 weight taps, tap (dy, dx) at position 3 dx + dy, so that for each
        // dx the three dy taps form one B operand of 3 COUT rows: 64 input
        // channels come by TMA in the producer (swizzled rows); fewer, from the
        // epilogue warps in the interleaved K-major core-matrix layout
        if (!S::SW) {
            for (int q = tid; q < 9 * COUT * (CIN / 8); q += 32 * EW) {
                const int t = q / (COUT * (CIN / 8)), rem = q - t * (COUT * (CIN / 8));
                const int n = rem / (CIN / 8), j = rem - n * (CIN / 8);
                const int pos = 3 * (t % 3) + t / 3;
                tc::cp_async16(sB + pos * S::B_TAP + tc::kmajor_offset(n, 8 * j, CIN),
                               a.w + ((int64_t)t * COUT + n) * CIN + 8 * j);
            }
            tc::cp_async_commit_wait_all();
            tc::fence_proxy_async();
            __syncwarp();
            if (lane == 0) tc::mbar_arrive(wbar);
        }
        // epilogue: thread = pixel (TMEM lane) x 16 channels
        const uint32_t lane_base = (uint32_t)((warp & 3) * 32) << 16;
        const int part = warp >> 2;
        const int pix = tid & 127;
        const int c0 = part * CPP;
        float bz[16];
#pragma unroll
        for (int i = 0; i < 16; ++i) bz[i] = (a.bias && part < PARTS) ? a.bias[c0 + i] : 0.f;
        uint32_t r = 0, ld0 = 0;
        bool ok = true;
        for (int64_t q = r0; q < r1 && ok;) {
            const ConvSeg g = conv_segment(q, r1, NY, ncb);
            for (int y = g.ya; y < g.yb; ++y, ++r) {
                const uint32_t kr = ld0 + (uint32_t)(y - g.ya) + 1;   // load of padded row y + 1
                const int x = g.x0 + pix;
                const int64_t po = pix_off(g.b, y, x, NY, NX);
                // residual and mask loads issued before the wait for the row's MMAs
                uint4 rp[2] = {}, mp[2] = {};
                if (a.resid && !ring_res) {
                    const uint4* rs = reinterpret_cast<const uint4*>(a.resid + po * COUT + c0);
                    rp[0] = rs[0];
                    rp[1] = rs[1];
                }
                if (a.mask) {
                    const uint4* ms = reinterpret_cast<const uint4*>(a.mask + po * COUT + c0);
                    mp[0] = ms[0];
                    mp[1] = ms[1];
                }
                const uint32_t acc = (0u - r) % (uint32_t)S::NACC;   // the row's TMEM slot
                const bool w = tc::mbar_wait_or_abort(&accf[acc], (r / S::NACC) & 1, abort_flag);
                if (!__all_sync(0xffffffffu, w)) { ok = false; break; }
                tc::fence_after_sync();
                float v[16];
                tc::tmem_ld16(tmem + lane_base + acc * COUT + (uint32_t)c0, v);
                tc::fence_before_sync();
                __syncwarp();
                if (lane == 0) tc::mbar_arrive(&acce[acc]);
                if (ring_res) {   // the residual from the ring slot of padded row y + 1
                    const uint32_t sl = kr % S::NSLOT;
                    const bool wr = tc::mbar_wait_or_abort(&full[sl], (kr / S::NSLOT) & 1, abort_flag);
                    if (!__all_sync(0xffffffffu, wr)) { ok = false; break; }
                    const unsigned char* row = sR + sl * S::ROW_BYTES;
                    const int px = pix + 1;
                    if (S::SW) {   // swizzled pixel row
                        rp[0] = *reinterpret_cast<const uint4*>(row + px * 128 + (((c0 / 8) ^ (px & 7)) * 16));
                        rp[1] = *reinterpret_cast<const uint4*>(row + px * 128 + (((c0 / 8 + 1) ^ (px & 7)) * 16));
                    } else {
                        rp[0] = *reinterpret_cast<const uint4*>(row + (c0 / 8) * S::LBO_A + px * 16);
                        rp[1] = *reinterpret_cast<const uint4*>(row + (c0 / 8 + 1) * S::LBO_A + px * 16);
                    }
                    __syncwarp();
                    if (lane == 0) tc::mbar_arrive(&empty[sl]);
                }
#pragma unroll
                for (int i = 0; i < 16; ++i) v[i] += bz[i];
                if (a.y4 && c0 == 0) {
                    const int64_t q4 = (((int64_t)g.b * NY + y) * NX + x) * 4;
#pragma unroll
                    for (int i = 0; i < 4; ++i) a.y4[q4 + i] = a.x4[q4 + i] + v[i];
                }
                __align__(16) __nv_bfloat16 hz[16], ho[16], hm[16];
                if (a.zout)
#pragma unroll
                    for (int i = 0; i < 16; ++i) hz[i] = __float2bfloat16_rn(v[i]);
                if (a.relu)
#pragma unroll
                    for (int i = 0; i < 16; ++i) v[i] = fmaxf(v[i], 0.f);
                if (a.resid) {
                    __align__(16) __nv_bfloat16 rr[16];
                    reinterpret_cast<uint4*>(rr)[0] = rp[0];
                    reinterpret_cast<uint4*>(rr)[1] = rp[1];
#pragma unroll
                    for (int i = 0; i < 16; ++i) v[i] += __bfloat162float(rr[i]);
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
                const bool halo_hi = (x == 0), halo_lo = (x == NX - 1);   // copies into columns NX + 1 / 0
                const int64_t po_h = halo_hi ? pix_off(g.b, y, NX, NY, NX) : pix_off(g.b, y, -1, NY, NX);
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
            ld0 += (uint32_t)(g.yb - g.ya) + 2;
            q += g.yb - g.ya;
        }
    }
    tc::fence_before_sync();
    __syncthreads();
    if (tid == 0 && *abort_flag) atomicExch(a.err, 1);
    if (warp == 0) tc::tmem_dealloc(tmem, S::TMEM_COLS);
}

// cuTensorMapEncodeTiled from the driver, found once through the runtime
typedef CUresult (*EncodeTiledFn)(CUtensorMap*, CUtensorMapDataType, cuuint32_t, void*, const cuuint64_t*,
                                  const cuuint64_t*, const cuuint32_t*, const cuuint32_t*, CUtensorMapInterleave,
                                  CUtensorMapSwizzle, CUtensorMapL2promotion, CUtensorMapFloatOOBfill);
static EncodeTiledFn encode_tiled()
{
    static const EncodeTiledFn fn = [] {
        void* p = nullptr;
        cudaDriverEntryPointQueryResult q{};
        if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault, &q) !=
                cudaSuccess ||
            q != cudaDriverEntryPointSuccess)
            return (EncodeTiledFn) nullptr;
        return (EncodeTiledFn)p;
    }();
    return fn;
}

template <int CIN, int COUT>
cudaError_t launch_conv(const ConvArgs& a, cudaStream_t s)
{
    using S = ConvSmem<CIN, COUT>;
    static unsigned long long attr_done = 0;      // per instantiation and device
    if (cudaError_t e = raise_smem_limit(k_conv3x3<CIN, COUT>, (int)S::BYTES, &attr_done); e != cudaSuccess) return e;
    const EncodeTiledFn enc = encode_tiled();
    if (!enc) return cudaErrorNotSupported;
    // the padded input as [B (NY + 2)][NX + 2][CIN]; a box is 130 pixels of one row, all 64 channels
    // (128-byte swizzle) or 8 channels
    CUtensorMap m;
    const cuuint64_t dims[3] = {(cuuint64_t)CIN, (cuuint64_t)a.NX + 2, (cuuint64_t)a.B * (a.NY + 2)};
    const cuuint64_t strides[2] = {(cuuint64_t)CIN * 2, (cuuint64_t)(a.NX + 2) * CIN * 2};
    const cuuint32_t box[3] = {S::SW ? (cuuint32_t)CIN : 8u, (cuuint32_t)S::RP, 1};
    const cuuint32_t estr[3] = {1, 1, 1};
    if (enc(&m, CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 3, const_cast<__nv_bfloat16*>(a.in), dims, strides, box, estr,
            CU_TENSOR_MAP_INTERLEAVE_NONE, S::SW ? CU_TENSOR_MAP_SWIZZLE_128B : CU_TENSOR_MAP_SWIZZLE_NONE,
            CU_TENSOR_MAP_L2_PROMOTION_L2_128B,
            CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) != CUDA_SUCCESS)
        return cudaErrorInvalidValue;
    // the weights as [9][COUT][CIN]; a box is one tap (used with 64 input channels)
    CUtensorMap mw;
    const cuuint64_t wdims[3] = {(cuuint64_t)CIN, (cuuint64_t)COUT, 9};
    const cuuint64_t wstrides[2] = {(cuuint64_t)CIN * 2, (cuuint64_t)COUT * CIN * 2};
    const cuuint32_t wbox[3] = {(cuuint32_t)CIN, (cuuint32_t)COUT, 1};
    if (enc(&mw, CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 3, const_cast<__nv_bfloat16*>(a.w), wdims, wstrides, wbox, estr,
            CU_TENSOR_MAP_INTERLEAVE_NONE, S::SW ? CU_TENSOR_MAP_SWIZZLE_128B : CU_TENSOR_MAP_SWIZZLE_NONE,
            CU_TENSOR_MAP_L2_PROMOTION_L2_128B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) != CUDA_SUCCESS)
        return cudaErrorInvalidValue;
    int sms = 0;
    if (cudaError_t e = device_sms(&sms); e != cudaSuccess) return e;
    const int64_t rows = (int64_t)a.B * (a.NX / 128) * a.NY;
    const int blocks = (int)(rows < sms ? rows : sms);
    k_conv3x3<CIN, COUT><<<blocks, conv_threads<COUT>(), S::BYTES, s>>>(m, mw, a);
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
// a GEMM over pixels (K) per tap, with the 64-channel side as M = 64 (i for
// CIN = 64, else o) and the other as N.  A work item is a slice of the row
// tiles (128 pixels of one image row) for one group of taps; it accumulates
// all of its rows in TMEM and writes one FP32 partial [tap][M][N], summed over
// the items by k_wgrad_reduce.  For 64 -> 64 the taps are split in three
// groups by dy; otherwise one group holds all nine.  The kernels below
// (k_wgrad64, k_wgrad16, k_wgrad_o16) stream the rows by TMA in swizzled
// MN-major layouts, where the tap shift dx is a 128- or 32-byte move of a
// descriptor start or of an M / N atom.
// ---------------------------------------------------------------------------
template <int CIN, int COUT>
struct WgCfg {
    static constexpr bool HA = CIN == 64;                  // h is the M = 64 operand of the partial
    static constexpr int NB = HA ? COUT : CIN;             // N of the partial
    static constexpr int NG = (CIN == 64 && COUT == 64) ? 3 : 1;
    static constexpr int TG = 9 / NG;                      // taps per group
    static constexpr int SLICES = (2 * 152) / NG;          // items per group
    static constexpr size_t PART = (size_t)NG * SLICES * TG * 64 * NB;   // floats
};

struct WgArgs {
    const __nv_bfloat16* h;      // padded NHWC CIN
    const __nv_bfloat16* g;      // padded NHWC COUT
    float* part;                 // [NG][SLICES][TG][64][NB]
    int B, NY, NX;
    int* err;
};

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

// ---------------------------------------------------------------------------
// Weight gradient of the 64 -> 64 convolution as a warp pipeline over the
// items of WgCfg<64, 64> (three tap groups by dy, each over a slice of the row
// tiles, partials [tap][i][o]); per row tile the producer warp
// brings g (128 pixels) and the h row of the group's dy (130 pixels) by TMA in
// the 128-byte swizzled layout, which is MN-major for this GEMM (a pixel is a
// K row of 64 channels).  The MMA warp takes M = 64 from g (output channel o)
// and N = 192 from h: the three dx taps stacked as the three 64-channel atoms
// of the B operand, one pixel (128 bytes) apart, so one MMA per 16 pixels
// covers the group's three taps.  Two TMEM accumulators of 192 columns let
// the epilogue warps write one item's partial while the next accumulates.
// ---------------------------------------------------------------------------
struct Wg64 {
    static constexpr int NSLOT = 6;
    static constexpr int G_BYTES = 128 * 128, H_BYTES = 17 * 1024;   // 128 / 130 pixel rows of 128 bytes
    static constexpr int SLOT = G_BYTES + H_BYTES;
    static constexpr int BAR_OFF = NSLOT * SLOT;
    static constexpr int NBAR = 2 * NSLOT + 2 + 2 + 1;                // full, empty, acc full, acc empty, done
    static constexpr int BYTES = BAR_OFF + NBAR * 8 + 16;
    static constexpr int THREADS = 6 * 32;                            // 4 epilogue warps, producer, MMA
    static_assert(SLOT % 1024 == 0 && G_BYTES % 1024 == 0, "swizzle patterns 1024-byte aligned");
};

__global__ void __launch_bounds__(Wg64::THREADS, 1)
    k_wgrad64(const __grid_constant__ CUtensorMap tg, const __grid_constant__ CUtensorMap th, WgArgs a)
{
    using S = WgCfg<64, 64>;
    using P = Wg64;
    extern __shared__ __align__(1024) unsigned char smem[];
    uint64_t* full = reinterpret_cast<uint64_t*>(smem + P::BAR_OFF);
    uint64_t* empty = full + P::NSLOT;
    uint64_t* accf = empty + P::NSLOT;
    uint64_t* acce = accf + 2;
    uint64_t* done = acce + 2;
    uint32_t* tslot = reinterpret_cast<uint32_t*>(done + 1);
    volatile int* abort_flag = reinterpret_cast<volatile int*>(tslot + 1);
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    const int NY = a.NY, NX = a.NX, ncb = NX / 128;
    const int64_t R = (int64_t)a.B * ncb * NY;
    constexpr int NITEM = S::NG * S::SLICES;
    static_assert(S::NG == 3 && S::TG == 3, "three tap groups by dy");

    if (warp == 0) tc::tmem_alloc(tslot, 512);
    if (tid == 0) {
        for (int i = 0; i < P::NSLOT; ++i) {
            tc::mbar_init(&full[i], 1);
            tc::mbar_init(&empty[i], 1);
        }
        for (int i = 0; i < 2; ++i) {
            tc::mbar_init(&accf[i], 1);
            tc::mbar_init(&acce[i], 4);
        }
        tc::mbar_init(done, 1);
        *abort_flag = (tc::smem_u32(smem) & 1023u) ? 1 : 0;
        tc::fence_mbar_init();
    }
    tc::fence_before_sync();
    __syncthreads();
    tc::fence_after_sync();
    const uint32_t tmem = *tslot;
    const bool start = *abort_flag == 0;
    // item `it` is tap group it mod 3 of slice it / 3, so that the three groups
    // of a slice run on neighbouring CTAs at the same time and share their g and
    // h rows in L2; its rows are [r0, r1) of the row tiles ordered (image,
    // column block, row), its partial sits at group * SLICES + slice
    auto item_rows = [&](int it, int64_t& r0, int64_t& r1) {
        const int sl = it / 3;
        r0 = R * sl / S::SLICES;
        r1 = R * (sl + 1) / S::SLICES;
    };

    if (warp == 4) {   // producer
        if (lane == 0 && start) {
            uint32_t ld = 0;
            bool ok = true;
            for (int it = blockIdx.x; it < NITEM && ok; it += gridDim.x) {
                const int gi = it % 3;                  // padded h row y + gi: dy = gi - 1
                int64_t r0, r1;
                item_rows(it, r0, r1);
                for (int64_t r = r0; r < r1; ++r, ++ld) {
                    const int64_t col = r / NY;
                    const int y = (int)(r - col * NY), b = (int)(col / ncb), x0 = (int)(col - (int64_t)b * ncb) * 128;
                    const uint32_t sl = ld % P::NSLOT;
                    if (!tc::mbar_wait_or_abort(&empty[sl], ((ld / P::NSLOT) & 1) ^ 1, abort_flag)) { ok = false; break; }
                    unsigned char* dst = smem + sl * P::SLOT;
                    tc::mbar_arrive_expect_tx(&full[sl], 128 * 128 + 130 * 128);
                    tc::tma_load_3d(dst, &tg, 0, x0 + 1, b * (NY + 2) + y + 1, &full[sl]);
                    tc::tma_load_3d(dst + P::G_BYTES, &th, 0, x0, b * (NY + 2) + y + gi, &full[sl]);
                }
            }
            for (uint32_t k = ld > (uint32_t)P::NSLOT ? ld - P::NSLOT : 0u; k < ld; ++k)
                tc::mbar_wait(&full[k % P::NSLOT], (k / P::NSLOT) & 1);
        }
    } else if (warp == 5) {   // MMA issue
        if (lane == 0 && start) {
            constexpr uint32_t idesc = tc::idesc_bf16_f32(64, 192) | (1u << 15) | (1u << 16);   // both MN-major
            const uint32_t base = tc::smem_u32(smem);
            uint32_t ld = 0, u = 0;
            bool ok = true, issued = false;
            for (int it = blockIdx.x; it < NITEM && ok; it += gridDim.x) {
                int64_t r0, r1;
                item_rows(it, r0, r1);
                if (r1 <= r0) continue;
                const uint32_t buf = u & 1, dcol = tmem + buf * 192;
                if (!tc::mbar_wait_or_abort(&acce[buf], ((u >> 1) & 1) ^ 1, abort_flag)) { ok = false; break; }
                tc::fence_after_sync();
                for (int64_t r = r0; r < r1; ++r, ++ld) {
                    const uint32_t sl = ld % P::NSLOT;
                    if (!tc::mbar_wait_or_abort(&full[sl], (ld / P::NSLOT) & 1, abort_flag)) { ok = false; break; }
                    tc::fence_after_sync();
                    const uint32_t gb = base + sl * P::SLOT, hb = gb + P::G_BYTES;
#pragma unroll
                    for (int s = 0; s < 8; ++s)   // 16 pixels per MMA
                        tc::mma_bf16(dcol, tc::smem_desc_sw128_mn(gb + s * 2048, 1024, 1024),
                                     tc::smem_desc_sw128_mn(hb + s * 2048, 128, 1024), idesc,
                                     (r == r0 && s == 0) ? 0u : 1u);
                    issued = true;
                    tc::mma_commit(&empty[sl]);
                }
                if (!ok) break;
                tc::mma_commit(&accf[buf]);
                ++u;
            }
            if (issued) {
                tc::mma_commit(done);
                tc::mbar_wait(done, 0);
            }
        }
    } else if (start) {   // epilogue: M = 64 rows 16 w + l sit in lanes 32 w + l, l < 16
        uint32_t u = 0;
        const int m = 16 * warp + lane;   // output channel o
        for (int it = blockIdx.x; it < NITEM; it += gridDim.x) {
            int64_t r0, r1;
            item_rows(it, r0, r1);
            float* dst = a.part + (size_t)((it % 3) * S::SLICES + it / 3) * 3 * 64 * 64;   // [tap j][i][o]
            if (r1 <= r0) {
                for (int q = lane; q < 3 * 64 * 16; q += 32) {   // this warp's 16 output channels
                    const int j = q / (64 * 16), rem = q - j * 64 * 16;
                    dst[((size_t)j * 64 + rem / 16) * 64 + 16 * warp + rem % 16] = 0.f;
                }
                continue;
            }
            const uint32_t buf = u & 1;
            const bool w = tc::mbar_wait_or_abort(&accf[buf], (u >> 1) & 1, abort_flag);
            if (!__all_sync(0xffffffffu, w)) break;
            tc::fence_after_sync();
#pragma unroll 1
            for (int j = 0; j < 3; ++j)
#pragma unroll 1
                for (int c0 = 0; c0 < 64; c0 += 16) {
                    float v[16];
                    tc::tmem_ld16(tmem + ((uint32_t)(warp * 32) << 16) + buf * 192 + (uint32_t)(j * 64 + c0), v);
                    if (lane < 16)
#pragma unroll
                        for (int q = 0; q < 16; ++q) dst[((size_t)j * 64 + c0 + q) * 64 + m] = v[q];
                }
            tc::fence_before_sync();
            __syncwarp();
            if (lane == 0) tc::mbar_arrive(&acce[buf]);
            ++u;
        }
    }
    tc::fence_before_sync();
    __syncthreads();
    if (tid == 0 && *abort_flag) atomicExch(a.err, 1);
    if (warp == 0) tc::tmem_dealloc(tmem, 512);
}

cudaError_t launch_wgrad64(const __nv_bfloat16* h, const __nv_bfloat16* g, int B, int NY, int NX, float* part,
                           size_t part_floats, float* dW, int* err, cudaStream_t s)
{
    using S = WgCfg<64, 64>;
    static unsigned long long attr_done = 0;
    if (cudaError_t e = raise_smem_limit(k_wgrad64, (int)Wg64::BYTES, &attr_done); e != cudaSuccess) return e;
    if (part_floats < S::PART) return cudaErrorInvalidValue;
    const EncodeTiledFn enc = encode_tiled();
    if (!enc) return cudaErrorNotSupported;
    // g and h as [B (NY + 2)][NX + 2][64], boxes of 128 / 130 pixels x 64 channels, 128-byte swizzle
    CUtensorMap mg, mh;
    const cuuint64_t dims[3] = {64, (cuuint64_t)NX + 2, (cuuint64_t)B * (NY + 2)};
    const cuuint64_t strides[2] = {128, (cuuint64_t)(NX + 2) * 128};
    const cuuint32_t boxg[3] = {64, 128, 1}, boxh[3] = {64, 130, 1}, estr[3] = {1, 1, 1};
    if (enc(&mg, CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 3, const_cast<__nv_bfloat16*>(g), dims, strides, boxg, estr,
            CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_128B, CU_TENSOR_MAP_L2_PROMOTION_L2_128B,
            CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) != CUDA_SUCCESS ||
        enc(&mh, CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 3, const_cast<__nv_bfloat16*>(h), dims, strides, boxh, estr,
            CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_128B, CU_TENSOR_MAP_L2_PROMOTION_L2_128B,
            CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) != CUDA_SUCCESS)
        return cudaErrorInvalidValue;
    int sms = 0;
    if (cudaError_t e = device_sms(&sms); e != cudaSuccess) return e;
    constexpr int NITEM = S::NG * S::SLICES;
    WgArgs a{h, g, part, B, NY, NX, err};
    k_wgrad64<<<NITEM < sms ? NITEM : sms, Wg64::THREADS, Wg64::BYTES, s>>>(mg, mh, a);
    const int n = 9 * 64 * 64;
    k_wgrad_reduce<64, 64><<<(n + 255) / 256, 256, 0, s>>>(part, dW);
    return cudaGetLastError();
}

// The 16 -> 64 weight gradient in the same form: h has 16 channels (32-byte
// rows, 32-byte swizzle), so a row tile's three h rows (dy = -1, 0, 1) come
// with its g row, and per 16 pixels one M = 64 x N = 48 MMA per dy covers the
// three dx taps (B atoms of 16 channels one pixel apart).  An item is a slice
// of row tiles with all nine taps (columns 16 t + i of a 144-column
// accumulator), partials [tap][o][i].
struct Wg16 {
    static constexpr int NSLOT = 6;
    static constexpr int G_BYTES = 128 * 128, H_ROW = 5 * 1024;       // g: 128 x 128 B; h: 130 x 32 B, padded
    static constexpr int SLOT = G_BYTES + 3 * H_ROW;
    static constexpr int TX = G_BYTES + 3 * 130 * 32;
    static constexpr int BAR_OFF = NSLOT * SLOT;
    static constexpr int NBAR = 2 * NSLOT + 2 + 2 + 1;
    static constexpr int BYTES = BAR_OFF + NBAR * 8 + 16;
    static constexpr int THREADS = 6 * 32;
    static_assert(SLOT % 1024 == 0 && G_BYTES % 1024 == 0 && H_ROW % 1024 == 0, "swizzle patterns aligned");
};

__global__ void __launch_bounds__(Wg16::THREADS, 1)
    k_wgrad16(const __grid_constant__ CUtensorMap tg, const __grid_constant__ CUtensorMap th, WgArgs a)
{
    using S = WgCfg<16, 64>;
    using P = Wg16;
    static_assert(S::NG == 1 && S::TG == 9 && S::NB == 16, "one item group of nine taps, 16 columns each");
    extern __shared__ __align__(1024) unsigned char smem[];
    uint64_t* full = reinterpret_cast<uint64_t*>(smem + P::BAR_OFF);
    uint64_t* empty = full + P::NSLOT;
    uint64_t* accf = empty + P::NSLOT;
    uint64_t* acce = accf + 2;
    uint64_t* done = acce + 2;
    uint32_t* tslot = reinterpret_cast<uint32_t*>(done + 1);
    volatile int* abort_flag = reinterpret_cast<volatile int*>(tslot + 1);
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    const int NY = a.NY, NX = a.NX, ncb = NX / 128;
    const int64_t R = (int64_t)a.B * ncb * NY;
    constexpr int NITEM = S::SLICES;

    if (warp == 0) tc::tmem_alloc(tslot, 512);
    if (tid == 0) {
        for (int i = 0; i < P::NSLOT; ++i) {
            tc::mbar_init(&full[i], 1);
            tc::mbar_init(&empty[i], 1);
        }
        for (int i = 0; i < 2; ++i) {
            tc::mbar_init(&accf[i], 1);
            tc::mbar_init(&acce[i], 4);
        }
        tc::mbar_init(done, 1);
        *abort_flag = (tc::smem_u32(smem) & 1023u) ? 1 : 0;
        tc::fence_mbar_init();
    }
    tc::fence_before_sync();
    __syncthreads();
    tc::fence_after_sync();
    const uint32_t tmem = *tslot;
    const bool start = *abort_flag == 0;

    if (warp == 4) {   // producer
        if (lane == 0 && start) {
            uint32_t ld = 0;
            bool ok = true;
            for (int it = blockIdx.x; it < NITEM && ok; it += gridDim.x) {
                const int64_t r0 = R * it / NITEM, r1 = R * (it + 1) / NITEM;
                for (int64_t r = r0; r < r1; ++r, ++ld) {
                    const int64_t col = r / NY;
                    const int y = (int)(r - col * NY), b = (int)(col / ncb), x0 = (int)(col - (int64_t)b * ncb) * 128;
                    const uint32_t sl = ld % P::NSLOT;
                    if (!tc::mbar_wait_or_abort(&empty[sl], ((ld / P::NSLOT) & 1) ^ 1, abort_flag)) { ok = false; break; }
                    unsigned char* dst = smem + sl * P::SLOT;
                    tc::mbar_arrive_expect_tx(&full[sl], P::TX);
                    tc::tma_load_3d(dst, &tg, 0, x0 + 1, b * (NY + 2) + y + 1, &full[sl]);
                    for (int d = 0; d < 3; ++d)   // padded h rows y, y + 1, y + 2 (dy = d - 1)
                        tc::tma_load_3d(dst + P::G_BYTES + d * P::H_ROW, &th, 0, x0, b * (NY + 2) + y + d, &full[sl]);
                }
            }
            for (uint32_t k = ld > (uint32_t)P::NSLOT ? ld - P::NSLOT : 0u; k < ld; ++k)
                tc::mbar_wait(&full[k % P::NSLOT], (k / P::NSLOT) & 1);
        }
    } else if (warp == 5) {   // MMA issue
        if (lane == 0 && start) {
            constexpr uint32_t idesc = tc::idesc_bf16_f32(64, 48) | (1u << 15) | (1u << 16);   // both MN-major
            const uint32_t base = tc::smem_u32(smem);
            uint32_t ld = 0, u = 0;
            bool ok = true, issued = false;
            for (int it = blockIdx.x; it < NITEM && ok; it += gridDim.x) {
                const int64_t r0 = R * it / NITEM, r1 = R * (it + 1) / NITEM;
                if (r1 <= r0) continue;
                const uint32_t buf = u & 1, dcol = tmem + buf * 144;
                if (!tc::mbar_wait_or_abort(&acce[buf], ((u >> 1) & 1) ^ 1, abort_flag)) { ok = false; break; }
                tc::fence_after_sync();
                for (int64_t r = r0; r < r1; ++r, ++ld) {
                    const uint32_t sl = ld % P::NSLOT;
                    if (!tc::mbar_wait_or_abort(&full[sl], (ld / P::NSLOT) & 1, abort_flag)) { ok = false; break; }
                    tc::fence_after_sync();
                    const uint32_t gb = base + sl * P::SLOT, hb = gb + P::G_BYTES;
#pragma unroll
                    for (int d = 0; d < 3; ++d)
#pragma unroll
                        for (int s = 0; s < 8; ++s)   // 16 pixels per MMA
                            tc::mma_bf16(dcol + 48 * d, tc::smem_desc_sw128_mn(gb + s * 2048, 1024, 1024),
                                         tc::smem_desc_sw32_mn(hb + d * P::H_ROW + s * 512, 32, 256), idesc,
                                         (r == r0 && s == 0) ? 0u : 1u);
                    issued = true;
                    tc::mma_commit(&empty[sl]);
                }
                if (!ok) break;
                tc::mma_commit(&accf[buf]);
                ++u;
            }
            if (issued) {
                tc::mma_commit(done);
                tc::mbar_wait(done, 0);
            }
        }
    } else if (start) {   // epilogue: M = 64 rows 16 w + l sit in lanes 32 w + l, l < 16
        uint32_t u = 0;
        const int o = 16 * warp + lane;
        for (int it = blockIdx.x; it < NITEM; it += gridDim.x) {
            const int64_t r0 = R * it / NITEM, r1 = R * (it + 1) / NITEM;
            float* dst = a.part + (size_t)it * 9 * 64 * 16;   // [tap][o][i]
            if (r1 <= r0) {
                for (int q = lane; q < 9 * 16 * 16; q += 32) {   // this warp's 16 output channels
                    const int t = q / 256, rem = q - t * 256;
                    dst[((size_t)t * 64 + 16 * warp + rem / 16) * 16 + rem % 16] = 0.f;
                }
                continue;
            }
            const uint32_t buf = u & 1;
            const bool w = tc::mbar_wait_or_abort(&accf[buf], (u >> 1) & 1, abort_flag);
            if (!__all_sync(0xffffffffu, w)) break;
            tc::fence_after_sync();
#pragma unroll 1
            for (int t = 0; t < 9; ++t) {
                float v[16];
                tc::tmem_ld16(tmem + ((uint32_t)(warp * 32) << 16) + buf * 144 + (uint32_t)(16 * t), v);
                if (lane < 16) {
                    float4* d4 = reinterpret_cast<float4*>(dst + ((size_t)t * 64 + o) * 16);
#pragma unroll
                    for (int q = 0; q < 4; ++q) d4[q] = make_float4(v[4 * q], v[4 * q + 1], v[4 * q + 2], v[4 * q + 3]);
                }
            }
            tc::fence_before_sync();
            __syncwarp();
            if (lane == 0) tc::mbar_arrive(&acce[buf]);
            ++u;
        }
    }
    tc::fence_before_sync();
    __syncthreads();
    if (tid == 0 && *abort_flag) atomicExch(a.err, 1);
    if (warp == 0) tc::tmem_dealloc(tmem, 512);
}

cudaError_t launch_wgrad16(const __nv_bfloat16* h, const __nv_bfloat16* g, int B, int NY, int NX, float* part,
                           size_t part_floats, float* dW, int* err, cudaStream_t s)
{
    using S = WgCfg<16, 64>;
    static unsigned long long attr_done = 0;
    if (cudaError_t e = raise_smem_limit(k_wgrad16, (int)Wg16::BYTES, &attr_done); e != cudaSuccess) return e;
    if (part_floats < S::PART) return cudaErrorInvalidValue;
    const EncodeTiledFn enc = encode_tiled();
    if (!enc) return cudaErrorNotSupported;
    // g as [B (NY + 2)][NX + 2][64] (boxes of 128 pixels, 128-byte swizzle); h with 16 channels (130 pixels, 32-byte)
    CUtensorMap mg, mh;
    const cuuint64_t gdims[3] = {64, (cuuint64_t)NX + 2, (cuuint64_t)B * (NY + 2)};
    const cuuint64_t gstr[2] = {128, (cuuint64_t)(NX + 2) * 128};
    const cuuint64_t hdims[3] = {16, (cuuint64_t)NX + 2, (cuuint64_t)B * (NY + 2)};
    const cuuint64_t hstr[2] = {32, (cuuint64_t)(NX + 2) * 32};
    const cuuint32_t boxg[3] = {64, 128, 1}, boxh[3] = {16, 130, 1}, estr[3] = {1, 1, 1};
    if (enc(&mg, CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 3, const_cast<__nv_bfloat16*>(g), gdims, gstr, boxg, estr,
            CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_128B, CU_TENSOR_MAP_L2_PROMOTION_L2_128B,
            CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) != CUDA_SUCCESS ||
        enc(&mh, CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 3, const_cast<__nv_bfloat16*>(h), hdims, hstr, boxh, estr,
            CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_32B, CU_TENSOR_MAP_L2_PROMOTION_L2_128B,
            CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) != CUDA_SUCCESS)
        return cudaErrorInvalidValue;
    int sms = 0;
    if (cudaError_t e = device_sms(&sms); e != cudaSuccess) return e;
    WgArgs a{h, g, part, B, NY, NX, err};
    k_wgrad16<<<S::SLICES < sms ? S::SLICES : sms, Wg16::THREADS, Wg16::BYTES, s>>>(mg, mh, a);
    const int n = 9 * 64 * 16;
    k_wgrad_reduce<16, 64><<<(n + 255) / 256, 256, 0, s>>>(part, dW);
    return cudaGetLastError();
}

// The 64 -> 16 weight gradient in the same form: here the shifted operand h
// (64 channels) is the M side, so per dy group and 16 pixels the taps
// dx = -1, 0 go into one M = 128 MMA (two M atoms one pixel apart; TMEM lanes
// 0-63 and 64-127) and dx = +1 into one M = 64 MMA, N = 16 output channels
// from g (32-byte swizzle).  A row tile's three h rows come with its g row;
// partials [tap][i][o].
struct WgO16 {
    static constexpr int NSLOT = 3;
    static constexpr int G_BYTES = 4096, H_ROW = 17 * 1024;           // g: 128 x 32 B; h: 130 x 128 B, padded
    static constexpr int SLOT = G_BYTES + 3 * H_ROW;
    static constexpr int TX = 128 * 32 + 3 * 130 * 128;
    static constexpr int BAR_OFF = NSLOT * SLOT;
    static constexpr int NBAR = 2 * NSLOT + 2 + 2 + 1;
    static constexpr int BYTES = BAR_OFF + NBAR * 8 + 16;
    static constexpr int THREADS = 6 * 32;
    static_assert(SLOT % 1024 == 0 && G_BYTES % 1024 == 0 && H_ROW % 1024 == 0, "swizzle patterns aligned");
};

__global__ void __launch_bounds__(WgO16::THREADS, 1)
    k_wgrad_o16(const __grid_constant__ CUtensorMap tg, const __grid_constant__ CUtensorMap th, WgArgs a)
{
    using S = WgCfg<64, 16>;
    using P = WgO16;
    static_assert(S::NG == 1 && S::TG == 9 && S::NB == 16 && S::HA, "one item group of nine taps, [i][o] partials");
    extern __shared__ __align__(1024) unsigned char smem[];
    uint64_t* full = reinterpret_cast<uint64_t*>(smem + P::BAR_OFF);
    uint64_t* empty = full + P::NSLOT;
    uint64_t* accf = empty + P::NSLOT;
    uint64_t* acce = accf + 2;
    uint64_t* done = acce + 2;
    uint32_t* tslot = reinterpret_cast<uint32_t*>(done + 1);
    volatile int* abort_flag = reinterpret_cast<volatile int*>(tslot + 1);
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    const int NY = a.NY, NX = a.NX, ncb = NX / 128;
    const int64_t R = (int64_t)a.B * ncb * NY;
    constexpr int NITEM = S::SLICES;

    if (warp == 0) tc::tmem_alloc(tslot, 256);
    if (tid == 0) {
        for (int i = 0; i < P::NSLOT; ++i) {
            tc::mbar_init(&full[i], 1);
            tc::mbar_init(&empty[i], 1);
        }
        for (int i = 0; i < 2; ++i) {
            tc::mbar_init(&accf[i], 1);
            tc::mbar_init(&acce[i], 4);
        }
        tc::mbar_init(done, 1);
        *abort_flag = (tc::smem_u32(smem) & 1023u) ? 1 : 0;
        tc::fence_mbar_init();
    }
    tc::fence_before_sync();
    __syncthreads();
    tc::fence_after_sync();
    const uint32_t tmem = *tslot;
    const bool start = *abort_flag == 0;

    if (warp == 4) {   // producer
        if (lane == 0 && start) {
            uint32_t ld = 0;
            bool ok = true;
            for (int it = blockIdx.x; it < NITEM && ok; it += gridDim.x) {
                const int64_t r0 = R * it / NITEM, r1 = R * (it + 1) / NITEM;
                for (int64_t r = r0; r < r1; ++r, ++ld) {
                    const int64_t col = r / NY;
                    const int y = (int)(r - col * NY), b = (int)(col / ncb), x0 = (int)(col - (int64_t)b * ncb) * 128;
                    const uint32_t sl = ld % P::NSLOT;
                    if (!tc::mbar_wait_or_abort(&empty[sl], ((ld / P::NSLOT) & 1) ^ 1, abort_flag)) { ok = false; break; }
                    unsigned char* dst = smem + sl * P::SLOT;
                    tc::mbar_arrive_expect_tx(&full[sl], P::TX);
                    tc::tma_load_3d(dst, &tg, 0, x0 + 1, b * (NY + 2) + y + 1, &full[sl]);
                    for (int d = 0; d < 3; ++d)   // padded h rows y, y + 1, y + 2 (dy = d - 1)
                        tc::tma_load_3d(dst + P::G_BYTES + d * P::H_ROW, &th, 0, x0, b * (NY + 2) + y + d, &full[sl]);
                }
            }
            for (uint32_t k = ld > (uint32_t)P::NSLOT ? ld - P::NSLOT : 0u; k < ld; ++k)
                tc::mbar_wait(&full[k % P::NSLOT], (k / P::NSLOT) & 1);
        }
    } else if (warp == 5) {   // MMA issue
        if (lane == 0 && start) {
            constexpr uint32_t id128 = tc::idesc_bf16_f32(128, 16) | (1u << 15) | (1u << 16);   // both MN-major
            constexpr uint32_t id64 = tc::idesc_bf16_f32(64, 16) | (1u << 15) | (1u << 16);
            const uint32_t base = tc::smem_u32(smem);
            uint32_t ld = 0, u = 0;
            bool ok = true, issued = false;
            for (int it = blockIdx.x; it < NITEM && ok; it += gridDim.x) {
                const int64_t r0 = R * it / NITEM, r1 = R * (it + 1) / NITEM;
                if (r1 <= r0) continue;
                const uint32_t buf = u & 1, dcol = tmem + buf * 96;
                if (!tc::mbar_wait_or_abort(&acce[buf], ((u >> 1) & 1) ^ 1, abort_flag)) { ok = false; break; }
                tc::fence_after_sync();
                for (int64_t r = r0; r < r1; ++r, ++ld) {
                    const uint32_t sl = ld % P::NSLOT;
                    if (!tc::mbar_wait_or_abort(&full[sl], (ld / P::NSLOT) & 1, abort_flag)) { ok = false; break; }
                    tc::fence_after_sync();
                    const uint32_t gb = base + sl * P::SLOT, hb = gb + P::G_BYTES;
#pragma unroll
                    for (int d = 0; d < 3; ++d)
#pragma unroll
                        for (int s = 0; s < 8; ++s) {   // 16 pixels per MMA
                            const uint64_t bd = tc::smem_desc_sw32_mn(gb + s * 512, 32, 256);
                            const uint32_t ha = hb + d * P::H_ROW + s * 2048;
                            const uint32_t acc = (r == r0 && s == 0) ? 0u : 1u;
                            tc::mma_bf16(dcol + 32 * d, tc::smem_desc_sw128_mn(ha, 128, 1024), bd, id128, acc);
                            tc::mma_bf16(dcol + 32 * d + 16, tc::smem_desc_sw128_mn(ha + 256, 1024, 1024), bd, id64, acc);
                        }
                    issued = true;
                    tc::mma_commit(&empty[sl]);
                }
                if (!ok) break;
                tc::mma_commit(&accf[buf]);
                ++u;
            }
            if (issued) {
                tc::mma_commit(done);
                tc::mbar_wait(done, 0);
            }
        }
    } else if (start) {   // epilogue: warp w reads TMEM lanes 32 w .. 32 w + 31
        uint32_t u = 0;
        for (int it = blockIdx.x; it < NITEM; it += gridDim.x) {
            const int64_t r0 = R * it / NITEM, r1 = R * (it + 1) / NITEM;
            float* dst = a.part + (size_t)it * 9 * 64 * 16;   // [tap][i][o]
            if (r1 <= r0) {
                for (int q = tid; q < 9 * 64 * 16; q += 128) dst[q] = 0.f;
                continue;
            }
            const uint32_t buf = u & 1;
            const bool w = tc::mbar_wait_or_abort(&accf[buf], (u >> 1) & 1, abort_flag);
            if (!__all_sync(0xffffffffu, w)) break;
            tc::fence_after_sync();
            auto put = [&](int t, int i, const float* v) {
                float4* d4 = reinterpret_cast<float4*>(dst + ((size_t)t * 64 + i) * 16);
#pragma unroll
                for (int q = 0; q < 4; ++q) d4[q] = make_float4(v[4 * q], v[4 * q + 1], v[4 * q + 2], v[4 * q + 3]);
            };
#pragma unroll 1
            for (int d = 0; d < 3; ++d) {
                float v[16];
                // M = 128: row m = lane 32 w + l is tap dx = m / 64 - 1 of channel i = m mod 64
                tc::tmem_ld16(tmem + ((uint32_t)(warp * 32) << 16) + buf * 96 + (uint32_t)(32 * d), v);
                const int m = 32 * warp + lane;
                put(3 * d + m / 64, m % 64, v);
                // M = 64 (tap dx = +1): row m = 16 w + l sits in lane 32 w + l, l < 16
                tc::tmem_ld16(tmem + ((uint32_t)(warp * 32) << 16) + buf * 96 + (uint32_t)(32 * d + 16), v);
                if (lane < 16) put(3 * d + 2, 16 * warp + lane, v);
            }
            tc::fence_before_sync();
            __syncwarp();
            if (lane == 0) tc::mbar_arrive(&acce[buf]);
            ++u;
        }
    }
    tc::fence_before_sync();
    __syncthreads();
    if (tid == 0 && *abort_flag) atomicExch(a.err, 1);
    if (warp == 0) tc::tmem_dealloc(tmem, 256);
}

cudaError_t launch_wgrad_o16(const __nv_bfloat16* h, const __nv_bfloat16* g, int B, int NY, int NX, float* part,
                             size_t part_floats, float* dW, int* err, cudaStream_t s)
{
    using S = WgCfg<64, 16>;
    static unsigned long long attr_done = 0;
    if (cudaError_t e = raise_smem_limit(k_wgrad_o16, (int)WgO16::BYTES, &attr_done); e != cudaSuccess) return e;
    if (part_floats < S::PART) return cudaErrorInvalidValue;
    const EncodeTiledFn enc = encode_tiled();
    if (!enc) return cudaErrorNotSupported;
    // g with 16 channels (boxes of 128 pixels, 32-byte swizzle); h with 64 (130 pixels, 128-byte)
    CUtensorMap mg, mh;
    const cuuint64_t gdims[3] = {16, (cuuint64_t)NX + 2, (cuuint64_t)B * (NY + 2)};
    const cuuint64_t gstr[2] = {32, (cuuint64_t)(NX + 2) * 32};
    const cuuint64_t hdims[3] = {64, (cuuint64_t)NX + 2, (cuuint64_t)B * (NY + 2)};
    const cuuint64_t hstr[2] = {128, (cuuint64_t)(NX + 2) * 128};
    const cuuint32_t boxg[3] = {16, 128, 1}, boxh[3] = {64, 130, 1}, estr[3] = {1, 1, 1};
    if (enc(&mg, CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 3, const_cast<__nv_bfloat16*>(g), gdims, gstr, boxg, estr,
            CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_32B, CU_TENSOR_MAP_L2_PROMOTION_L2_128B,
            CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) != CUDA_SUCCESS ||
        enc(&mh, CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 3, const_cast<__nv_bfloat16*>(h), hdims, hstr, boxh, estr,
            CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_128B, CU_TENSOR_MAP_L2_PROMOTION_L2_128B,
            CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) != CUDA_SUCCESS)
        return cudaErrorInvalidValue;
    int sms = 0;
    if (cudaError_t e = device_sms(&sms); e != cudaSuccess) return e;
    WgArgs a{h, g, part, B, NY, NX, err};
    k_wgrad_o16<<<S::SLICES < sms ? S::SLICES : sms, WgO16::THREADS, WgO16::BYTES, s>>>(mg, mh, a);
    const int n = 9 * 16 * 64;
    k_wgrad_reduce<64, 16><<<(n + 255) / 256, 256, 0, s>>>(part, dW);
    return cudaGetLastError();
}

cudaError_t conv3x3_wgrad(int cin, int cout, const __nv_bfloat16* h, const __nv_bfloat16* g, int B, int NY, int NX,
                          float* part, size_t part_floats, float* dW, int* err, cudaStream_t s)
{
    if (cin == 16 && cout == 64) return launch_wgrad16(h, g, B, NY, NX, part, part_floats, dW, err, s);
    if (cin == 64 && cout == 64) return launch_wgrad64(h, g, B, NY, NX, part, part_floats, dW, err, s);
    if (cin == 64 && cout == 16) return launch_wgrad_o16(h, g, B, NY, NX, part, part_floats, dW, err, s);
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
