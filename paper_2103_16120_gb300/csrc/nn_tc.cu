// nn_tc.cu -- the 3x3 convolution of nn_conv.cu on the fifth-generation
// tensor cores (tcgen05): BF16 operands from shared memory, FP32 accumulator
// in tensor memory (TMEM), one thread issuing the MMAs.
//
// Tile: 128 consecutive output points of one latitude row (M = 128) x all
// output channels (N = COUT).  Operands use the no-swizzle K-major layout:
// 16-byte rows (8 channels) of consecutive points (or output channels), one
// plane per 8 input channels.  In this layout a longitude tap shift is a
// start-address offset of 16 bytes per point, so the nine taps read the
// staged halo rows directly: for tap (ky, kx) and input channels 16 ks ..
// 16 ks + 15, A starts at row ky, plane 2 ks, point kx, and one
// tcgen05.mma of K = 16 accumulates it.
//
// A block works down a strip of 16 rows of one 128-point column.  Input
// rows sit in a ring of four shared-memory slots (plus the two shifted pole
// rows of the input gradient), so every input row is staged once, and the
// accumulator is double-buffered in TMEM.  While the tensor core computes
// row h (thread 0 issues 9 * CIN / 16 MMAs, 12 * ... on a pole row, and
// commits them to an mbarrier), the block reads row h-1 out of TMEM
// (each warp its 32 lanes), stores it, and stages input row h+2 with
// cp.async into the slot row h-2 used.  Every mbarrier wait is bounded.
#include <cuda_bf16.h>
#include <cstdint>

#include "nn_internal.h"

namespace nn {

namespace {

constexpr int TC_TW = 128;                  // points per tile (MMA M)
constexpr int TC_P = TC_TW + 2;             // staged points per row (halo)
constexpr unsigned long long TC_WAIT_NS = 200000000ull;   // longest wait: 0.2 s

__device__ __forceinline__ unsigned smem_u32(const void *p) { return (unsigned)__cvta_generic_to_shared(p); }

__device__ __forceinline__ void cp16(void *s, const void *g)
{
    asm volatile("cp.async.cg.shared.global [%0], [%1], 16;" ::"r"(smem_u32(s)), "l"(g) : "memory");
}

__device__ __forceinline__ unsigned long long gtime()
{
    unsigned long long t;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
    return t;
}

// shared-memory matrix descriptor: start, leading (K) and stride (M/N)
// byte offsets in 16-byte units, descriptor version 1, no swizzle.  In both
// the K-major and the MN-major no-swizzle layouts the leading offset is the
// step between core matrices along K and the stride offset the step along
// M or N.
__device__ __forceinline__ unsigned long long sdesc(unsigned addr, unsigned lbo, unsigned sbo)
{
    return (unsigned long long)((addr & 0x3FFFF) >> 4) | ((unsigned long long)((lbo >> 4) & 0x3FFF) << 16) |
           ((unsigned long long)((sbo >> 4) & 0x3FFF) << 32) | (1ull << 46);
}

// instruction descriptor of kind::f16: FP32 accumulator, BF16 A and B, both
// K-major, N and M
__host__ __device__ constexpr unsigned idesc_bf16(int M, int N)
{
    return (1u << 4) | (1u << 7) | (1u << 10) | ((unsigned)(N >> 3) << 17) | ((unsigned)(M >> 4) << 24);
}

__device__ __forceinline__ void mma_bf16(unsigned dtmem, unsigned long long a, unsigned long long b, unsigned id,
                                         unsigned accumulate)
{
    asm volatile(
        "{\n .reg .pred p;\n setp.ne.u32 p, %4, 0;\n"
        " tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n}\n" ::"r"(dtmem),
        "l"(a), "l"(b), "r"(id), "r"(accumulate)
        : "memory");
}

__device__ __forceinline__ void mma_commit(unsigned mbar)
{
    asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(mbar)
                 : "memory");
}

// wait for the mbarrier phase of the given parity; false after TC_WAIT_NS
// (the clock is read every 64 polls)
__device__ __forceinline__ bool mbar_wait(unsigned mbar, unsigned parity)
{
    unsigned long long t0 = 0;
    for (unsigned n = 0;; ++n) {
        unsigned done;
        asm volatile(
            "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n"
            " selp.u32 %0, 1, 0, p;\n}\n"
            : "=r"(done)
            : "r"(mbar), "r"(parity)
            : "memory");
        if (done) return true;
        if ((n & 63) == 0) {
            const unsigned long long t = gtime();
            if (n == 0) t0 = t;
            else if (t - t0 > TC_WAIT_NS) return false;
        }
    }
}

__device__ __forceinline__ void tmem_ld8(unsigned taddr, float (&v)[8])
{
    unsigned r[8];
    asm volatile("tcgen05.ld.sync.aligned.32x32b.x8.b32 {%0,%1,%2,%3,%4,%5,%6,%7}, [%8];"
                 : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7])
                 : "r"(taddr));
#pragma unroll
    for (int q = 0; q < 8; ++q) v[q] = __uint_as_float(r[q]);
}

__host__ __device__ constexpr int tmem_cols(int n) { return n <= 32 ? 32 : (n <= 64 ? 64 : (n <= 128 ? 128 : 256)); }

} // namespace

constexpr int TC_STRIP = 8;                 // rows of one work unit
constexpr int TC_RING = 5;                  // ring slots of input rows
// ring of 5 input rows, plus 2 shifted pole rows for the input gradient
__host__ __device__ constexpr int tc_slots(bool dgrad) { return dgrad ? TC_RING + 2 : TC_RING; }

template <int CIN, int COUT, bool DGRAD>
__global__ void __launch_bounds__(128) k_conv_tc(ConvArgs a, int *err)
{
    constexpr int KC = CIN / 8;                 // 16-byte channel chunks of an input point
    constexpr unsigned TCOLS = tmem_cols(COUT);
    constexpr unsigned ID = idesc_bf16(TC_TW, COUT);
    constexpr int SLOT = KC * TC_P * 16;        // bytes of one staged row
    extern __shared__ __align__(1024) unsigned char smem[];
    unsigned char *Ws = smem;                                         // [9][KC][COUT] x 16 B
    unsigned char *Xs = Ws + (size_t)9 * KC * COUT * 16;              // [slot][KC][TC_P] x 16 B
    __shared__ __align__(8) unsigned long long s_mbar[2];
    __shared__ unsigned s_tmem;
    __shared__ int s_bad;
    __shared__ float s_bias[COUT];
    const int H = a.H, W = a.W;
    const int nseg = W / TC_TW;
    const int nstrip = (H + TC_STRIP - 1) / TC_STRIP;
    const long nunits = (long)a.B * nseg * nstrip;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;

    if (threadIdx.x == 0) {
        s_bad = 0;
        asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(smem_u32(&s_mbar[0])) : "memory");
        asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(smem_u32(&s_mbar[1])) : "memory");
    }
    if (warp == 0) {
        // two accumulators: the tensor core fills one while the other is read out
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(&s_tmem)),
                     "r"(2 * TCOLS)
                     : "memory");
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
    }
    for (int q = threadIdx.x; q < 9 * COUT * KC; q += blockDim.x) {
        const int c = q % KC, o = (q / KC) % COUT, tap = q / KC / COUT;
        cp16(Ws + ((size_t)(tap * KC + c) * COUT + o) * 16, a.w + ((size_t)tap * COUT + o) * CIN + c * 8);
    }
    for (int q = threadIdx.x; q < COUT; q += blockDim.x) s_bias[q] = a.bias ? a.bias[q] : 0.f;
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
    __syncthreads();
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
    const unsigned tmem = s_tmem;
    unsigned par[2] = {0, 0};

    // stage input row hs (with halo; shift: across-pole ghost) into a slot;
    // rows outside 0..H-1 give the sphere halo (forward) or zero (DGRAD)
    auto stage = [&](int slot, int b, int w0, int hr, bool pole_shift) {
        int hs = hr, shift = pole_shift ? W / 2 : 0;
        bool zero = false;
        if (!pole_shift && (hs < 0 || hs >= H)) {
            if (DGRAD) zero = true;
            else { hs = hs < 0 ? 0 : H - 1; shift = W / 2; }
        }
        unsigned char *base = Xs + (size_t)slot * SLOT;
        for (int q = threadIdx.x; q < TC_P * KC; q += blockDim.x) {
            const int c = q % KC, pt = q / KC;
            unsigned char *dst = base + ((size_t)c * TC_P + pt) * 16;
            if (zero) {
                *(uint4 *)dst = make_uint4(0, 0, 0, 0);
            } else {
                int ws = (w0 - 1 + pt + shift) % W;
                if (ws < 0) ws += W;
                cp16(dst, a.x + (((size_t)b * H + hs) * W + ws) * CIN + c * 8);
            }
        }
    };
    auto ready = [&]() {   // staged rows visible to the tensor core
        asm volatile("cp.async.wait_all;" ::: "memory");
        asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
        asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
        __syncthreads();
        asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
    };
    // read accumulator buf (row h of the unit) out of TMEM and store it
    auto epilogue = [&](int buf, int b, int h, int w0) {
        const int p = warp * 32 + lane;
        const size_t pix = ((size_t)b * H + h) * W + w0 + p;
        const unsigned trow = tmem + (unsigned)buf * TCOLS + ((unsigned)(warp * 32) << 16);
#pragma unroll
        for (int c0 = 0; c0 < COUT; c0 += 8) {
            float v[8];
            tmem_ld8(trow + c0, v);
            asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
#pragma unroll
            for (int q = 0; q < 8; ++q) {
                const int co = c0 + q;
                float x = v[q] + s_bias[co];
                if (a.relu) x = fmaxf(x, 0.f);
                if (a.mask && !(__bfloat162float(a.mask[pix * COUT + co]) > 0.f)) x = 0.f;
                v[q] = x;
            }
            if (a.yf) {
#pragma unroll
                for (int q = 0; q < 8; ++q)
                    if (c0 + q < a.yf_c) a.yf[pix * a.yf_c + c0 + q] = v[q];
            } else {
                __nv_bfloat162 o2[4];
#pragma unroll
                for (int q = 0; q < 4; ++q) o2[q] = __floats2bfloat162_rn(v[2 * q], v[2 * q + 1]);
                *(uint4 *)(a.y + pix * COUT + c0) = *(const uint4 *)o2;
            }
        }
    };
    auto wait_acc = [&](int buf) {
        const bool okw = mbar_wait(smem_u32(&s_mbar[buf]), par[buf]);
        par[buf] ^= 1;
        if (!okw && lane == 0) atomicExch(&s_bad, 1);
    };

    for (long unit = blockIdx.x; unit < nunits && !s_bad; unit += gridDim.x) {
        const int seg = (int)(unit % nseg);
        const int strip = (int)((unit / nseg) % nstrip);
        const int b = (int)(unit / nseg / nstrip);
        const int w0 = seg * TC_TW;
        const int h0 = strip * TC_STRIP, h1 = min(h0 + TC_STRIP, H);
        // ring: input row hr lives in slot (hr + TC_RING) % TC_RING; the
        // shifted pole rows (input gradient) in slots TC_RING and TC_RING + 1
        auto slot_of = [](int hr) { return (hr + TC_RING) % TC_RING; };
        for (int hr = h0 - 1; hr <= h0 + 1; ++hr) stage(slot_of(hr), b, w0, hr, false);
        if (DGRAD && h0 == 0) stage(TC_RING, b, w0, 0, true);
        if (DGRAD && h1 == H) stage(TC_RING + 1, b, w0, H - 1, true);
        ready();
        for (int h = h0; h < h1; ++h) {
            const int buf = (h - h0) & 1;
            // input row h+2 (for row h+1) goes into the slot that row h-3 held;
            // the last MMAs to read it were row h-2's, complete since the
            // previous iteration.  Its copy overlaps this iteration.
            if (h + 2 <= h1) stage(slot_of(h + 2), b, w0, h + 2, false);
            if (threadIdx.x == 0) {
                const unsigned xs = smem_u32(Xs), ws0 = smem_u32(Ws);
                const bool pole = DGRAD && (h == 0 || h == H - 1);
                const int ntap = pole ? 12 : 9;
                const unsigned d = tmem + (unsigned)buf * TCOLS;
                unsigned acc = 0;
                for (int t = 0; t < ntap; ++t) {
                    int tap, slot;
                    if (t < 9) { tap = t; slot = slot_of(h - 1 + t / 3); }
                    else { tap = (h == 0 ? 6 : 0) + (t - 9); slot = h == 0 ? TC_RING : TC_RING + 1; }
                    const int kx = tap % 3;
#pragma unroll
                    for (int ks = 0; ks < CIN / 16; ++ks) {
                        const unsigned aa = xs + (unsigned)slot * SLOT + ((unsigned)(2 * ks) * TC_P + kx) * 16;
                        const unsigned ba = ws0 + (unsigned)(tap * KC + 2 * ks) * COUT * 16;
                        mma_bf16(d, sdesc(aa, TC_P * 16, 128), sdesc(ba, COUT * 16, 128), ID, acc);
                        acc = 1;
                    }
                }
                mma_commit(smem_u32(&s_mbar[buf]));
            }
            __syncwarp();
            if (h > h0) {
                // row h-1: its MMAs are done once its barrier phase completes
                wait_acc(buf ^ 1);
                __syncthreads();
                if (s_bad) break;
                asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
                epilogue(buf ^ 1, b, h - 1, w0);
            }
            ready();      // row h+2 staged; accumulator buf ^ 1 free for row h+1
        }
        if (s_bad) break;
        // the unit's last row
        wait_acc((h1 - 1 - h0) & 1);
        __syncthreads();
        if (s_bad) break;
        asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
        epilogue((h1 - 1 - h0) & 1, b, h1 - 1, w0);
        asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
        __syncthreads();
        asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
    }
    if (s_bad && threadIdx.x == 0) {
        // a tensor-core wait ran out: flag it, and give outstanding work a
        // bounded chance to drain before TMEM is freed
        atomicExch(err, 1);
        mbar_wait(smem_u32(&s_mbar[0]), par[0]);
        mbar_wait(smem_u32(&s_mbar[1]), par[1]);
    }
    asm volatile("cp.async.wait_all;" ::: "memory");
    __syncthreads();
    if (warp == 0)
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(2 * TCOLS)
                     : "memory");
}

// ---------------------------------------------------------------------------
template <int CIN, int COUT, bool DGRAD>
static size_t tc_smem()
{
    return (size_t)9 * (CIN / 8) * COUT * 16 + (size_t)tc_slots(DGRAD) * (CIN / 8) * TC_P * 16;
}

template <int CIN, int COUT, bool DGRAD>
static cudaError_t conv_tc_t(const ConvArgs &a, int sms, int *err, cudaStream_t s)
{
    const size_t smem = tc_smem<CIN, COUT, DGRAD>();
    int bps = 0;
    cudaError_t e = occupancy_once<k_conv_tc<CIN, COUT, DGRAD>>(128, smem, &bps);
    if (e != cudaSuccess) return e;
    if (bps < 1) return cudaErrorInvalidConfiguration;
    // TMEM: 512 columns per SM shared by the resident blocks
    const int per = 2 * tmem_cols(COUT);
    if (bps * per > 512) bps = 512 / per;
    const long nunits = (long)a.B * (a.W / TC_TW) * ((a.H + TC_STRIP - 1) / TC_STRIP);
    long grid = (long)bps * sms;
    if (grid > nunits) grid = nunits;
    k_conv_tc<CIN, COUT, DGRAD><<<(int)grid, 128, smem, s>>>(a, err);
    return cudaGetLastError();
}

// true when the tcgen05 kernel takes this convolution: rows of a multiple of
// 128 points, operands within shared memory, and a layer where it measured
// faster than the mma.sync kernel (the forward layers with 32 or more input
// channels; with few MMAs per row, or a per-point FP32 store of many
// channels, the fixed cost per row dominates)
bool conv_tc_supported(int cin, int cout, bool dgrad, int W)
{
    if (W % TC_TW || dgrad || cin < 32 || cout < 32) return false;
    const size_t smem = (size_t)9 * (cin / 8) * cout * 16 + (size_t)tc_slots(dgrad) * (cin / 8) * TC_P * 16;
    if (smem > 227 * 1024) return false;
#define NN_TC(CI, CO) if (cin == CI && cout == CO) return true;
    NN_TC(16, 32) NN_TC(32, 64) NN_TC(96, 32) NN_TC(32, 16) NN_TC(64, 32) NN_TC(64, 128) NN_TC(32, 96)
    NN_TC(64, 64) NN_TC(128, 64)
#undef NN_TC
    return false;
}

cudaError_t launch_conv_tc(int cin, int cout, bool dgrad, const ConvArgs &a, int sms, int *err, cudaStream_t s)
{
#define NN_TC(CI, CO)                                                                            \
    if (cin == CI && cout == CO)                                                                 \
        return dgrad ? conv_tc_t<CI, CO, true>(a, sms, err, s) : conv_tc_t<CI, CO, false>(a, sms, err, s);
    NN_TC(16, 32) NN_TC(32, 64) NN_TC(96, 32) NN_TC(32, 16) NN_TC(64, 32) NN_TC(64, 128) NN_TC(32, 96)
    NN_TC(64, 64) NN_TC(128, 64)
#undef NN_TC
    return cudaErrorInvalidValue;
}

// ---------------------------------------------------------------------------
// weight gradient on tcgen05
// ---------------------------------------------------------------------------
// dW[ky][kx][co][ci] = sum over points p of x[row h + ky - 1][p + kx - 1][ci]
// g[row h][p][co], with the forward convolution's sphere halo.  As a GEMM
// D[m][n] = sum_k A[m][k] B[n][k]: m = ci (M = 128), n = co (N = COUT) for
// each tap, k = points.  The operands sit in shared memory in the layout the
// forward kernel stages (one plane per 8 channels, a 16-byte row per point),
// which for this GEMM is the MN-major no-swizzle layout (8 consecutive MN
// elements per 16-byte row, 8 rows per K core matrix): both are read with
// the transpose bits of the instruction descriptor set, and a longitude tap
// shift is a 16-byte start offset.  With fewer than 128 input channels the A
// operand's upper rows read the next ring slot: those rows of D are never
// read out.
//
// A block works down a strip of WG_STRIP output rows of one 128-point column
// and accumulates KYS kernel rows (3 KYS taps, 3 KYS COUT TMEM columns) over
// all of its strips; only at the end are the accumulators read out of TMEM
// and added to dW.  Input rows sit in a ring (each staged once per strip) and
// gradient rows in a second one, WG_AHEAD rows ahead of the MMAs; every row's
// MMAs are committed to one of three mbarriers, and a ring slot is restaged
// only after the MMAs of the last row that reads it are complete.  Every wait
// is bounded.
constexpr int WG_STRIP = 8;     // output rows of one work unit
constexpr int WG_AHEAD = 2;     // rows staged ahead of the MMAs

template <int CIN, int COUT, int KYS>
struct WgShape {
    static constexpr int KC = CIN / 8, GC = COUT / 8;
    static constexpr int XR = WG_AHEAD + KYS + 1;                  // input-row ring slots
    static constexpr int GR = WG_AHEAD + 2;                        // gradient-row ring slots
    static constexpr size_t XSLOT = (size_t)KC * TC_P * 16;
    static constexpr size_t XPAD = (size_t)(16 - KC) * TC_P * 16;  // the last slot's 16-plane read
    static constexpr size_t GSLOT = (size_t)GC * TC_TW * 16;
    static constexpr size_t BYTES = XR * XSLOT + XPAD + GR * GSLOT;
    static constexpr unsigned NCOL = 3 * KYS * COUT;
};

template <int CIN, int COUT, int KYS>
__global__ void __launch_bounds__(128) k_wgrad_tc(WgradArgs a, int *err)
{
    typedef WgShape<CIN, COUT, KYS> S;
    constexpr unsigned TCOLS = tmem_cols(S::NCOL);
    // BF16 A and B, both MN-major (transpose bits 15 and 16), FP32 accumulator
    constexpr unsigned ID = idesc_bf16(TC_TW, COUT) | (1u << 15) | (1u << 16);
    constexpr int NKG = 3 / KYS;                       // groups of kernel rows
    extern __shared__ __align__(1024) unsigned char smem[];
    unsigned char *Xs = smem, *Gs = smem + S::XR * S::XSLOT + S::XPAD;
    __shared__ __align__(8) unsigned long long s_mbar[3];
    __shared__ unsigned s_tmem;
    __shared__ int s_bad;
    const int H = a.H, W = a.W;
    const int nseg = W / TC_TW, nstrip = (H + WG_STRIP - 1) / WG_STRIP;
    const long nunits = (long)a.B * nseg * nstrip;
    const int ky0 = (blockIdx.x % NKG) * KYS;
    const int split = blockIdx.x / NKG, nsplit = gridDim.x / NKG;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const bool do_bias = a.db && ky0 == 0;

    if (threadIdx.x == 0) {
        s_bad = 0;
        for (int q = 0; q < 3; ++q)
            asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(smem_u32(&s_mbar[q])) : "memory");
    }
    if (warp == 0) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(&s_tmem)),
                     "r"(TCOLS)
                     : "memory");
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
    }
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
    __syncthreads();
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
    const unsigned tmem = s_tmem;
    unsigned par[3] = {0, 0, 0};
    bool pend[3] = {false, false, false};

    auto xslot = [&](int xr) { return Xs + (size_t)((xr + 2 * S::XR) % S::XR) * S::XSLOT; };
    auto gslot = [&](int h) { return Gs + (size_t)(h % S::GR) * S::GSLOT; };
    // input row xr (-1 .. H) with the sphere halo: beyond a pole, the pole row
    // shifted by half a circle
    auto stage_x = [&](int b, int w0, int xr) {
        int hs = xr, shift = 0;
        if (hs < 0) { hs = 0; shift = W / 2; }
        else if (hs >= H) { hs = H - 1; shift = W / 2; }
        unsigned char *xs = xslot(xr);
        for (int q = threadIdx.x; q < TC_P * S::KC; q += blockDim.x) {
            const int c = q % S::KC, pt = q / S::KC;
            int ws = (w0 - 1 + pt + shift) % W;
            if (ws < 0) ws += W;
            cp16(xs + ((size_t)c * TC_P + pt) * 16, a.x + (((size_t)b * H + hs) * W + ws) * CIN + c * 8);
        }
    };
    auto stage_g = [&](int b, int w0, int h) {
        unsigned char *gs = gslot(h);
        for (int q = threadIdx.x; q < TC_TW * S::GC; q += blockDim.x) {
            const int c = q % S::GC, pt = q / S::GC;
            cp16(gs + ((size_t)c * TC_TW + pt) * 16, a.g + (((size_t)b * H + h) * W + w0 + pt) * COUT + c * 8);
        }
    };
    // the MMAs committed to mbarrier q are complete
    auto wait_row = [&](int q) {
        if (!pend[q]) return;
        const bool okw = mbar_wait(smem_u32(&s_mbar[q]), par[q]);
        par[q] ^= 1;
        pend[q] = false;
        if (!okw && lane == 0) atomicExch(&s_bad, 1);
    };

    float bsum = 0.f;
    unsigned acc = 0;
    for (long u = split; u < nunits && !s_bad; u += nsplit) {
        const int seg = (int)(u % nseg);
        const int strip = (int)((u / nseg) % nstrip);
        const int b = (int)(u / nseg / nstrip);
        const int w0 = seg * TC_TW;
        const int h0 = strip * WG_STRIP, h1 = min(h0 + WG_STRIP, H);
        // the previous unit's MMAs read the slots about to be restaged
        for (int q = 0; q < 3; ++q) wait_row(q);
        __syncthreads();
        // prologue: the input and gradient rows of the first WG_AHEAD output rows
        const int hp = min(h0 + WG_AHEAD, h1);
        for (int xr = h0 + ky0 - 1; xr <= hp - 1 + ky0 + KYS - 2; ++xr) stage_x(b, w0, xr);
        for (int h = h0; h < hp; ++h) stage_g(b, w0, h);
        asm volatile("cp.async.commit_group;" ::: "memory");
        asm volatile("cp.async.wait_group 0;" ::: "memory");
        for (int h = h0; h < h1; ++h) {
            // rows for output row h + WG_AHEAD: its newest input row and its
            // gradient row, into the slots that output row h - 2 read last
            const int hn = h + WG_AHEAD;
            if (hn < h1) {
                if (h - 2 >= h0) wait_row((h - 2) % 3);
                __syncthreads();
                stage_x(b, w0, hn + ky0 + KYS - 2);
                stage_g(b, w0, hn);
            }
            asm volatile("cp.async.commit_group;" ::: "memory");
            // row h's copies were committed WG_AHEAD groups ago (or in the prologue)
            asm volatile("cp.async.wait_group %0;" ::"n"(WG_AHEAD) : "memory");
            asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
            asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
            __syncthreads();
            asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
            if (s_bad) break;
            wait_row(h % 3);                       // row h - 3 left this mbarrier's phase
            if (threadIdx.x == 0) {
                const unsigned ga = smem_u32(gslot(h));
#pragma unroll
                for (int kyl = 0; kyl < KYS; ++kyl) {
                    const unsigned xa = smem_u32(xslot(h + ky0 + kyl - 1));
#pragma unroll
                    for (int kx = 0; kx < 3; ++kx) {
#pragma unroll
                        for (int ks = 0; ks < TC_TW / 16; ++ks) {
                            const unsigned aa = xa + (unsigned)(ks * 16 + kx) * 16;
                            const unsigned ba = ga + (unsigned)(ks * 16) * 16;
                            // MN-major: the leading offset steps along K (8 points,
                            // 128 bytes), the stride offset along MN (one plane)
                            mma_bf16(tmem + (unsigned)((kyl * 3 + kx) * COUT), sdesc(aa, 128, TC_P * 16),
                                     sdesc(ba, 128, TC_TW * 16), ID, acc | (unsigned)ks);
                        }
                    }
                }
                mma_commit(smem_u32(&s_mbar[h % 3]));
            }
            __syncwarp();
            acc = 1;
            pend[h % 3] = true;
            if (do_bias) {
                // bias gradient: thread t adds channel t % COUT over every
                // (128 / COUT)-th point of the row, all threads at once
                constexpr int NPART = 128 / COUT;
                const unsigned char *gs = gslot(h);
                const int co = threadIdx.x % COUT, c = co / 8, e = co % 8;
#pragma unroll 8
                for (int p = threadIdx.x / COUT; p < TC_TW; p += NPART)
                    bsum += __bfloat162float(((const __nv_bfloat16 *)(gs + ((size_t)c * TC_TW + p) * 16))[e]);
            }
        }
    }
    for (int q = 0; q < 3; ++q) wait_row(q);
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
    __syncthreads();
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
    if (!s_bad && acc) {
        // lanes = input channels (warp w: 32 w .. 32 w + 31), columns = (ky, kx, co)
        const int ci = warp * 32 + lane;
        const unsigned trow = tmem + ((unsigned)(warp * 32) << 16);
#pragma unroll 4
        for (int c0 = 0; c0 < (int)S::NCOL; c0 += 8) {
            float v[8];
            tmem_ld8(trow + c0, v);
            asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
            if (ci < CIN) {
#pragma unroll
                for (int q = 0; q < 8; ++q) {
                    const int col = c0 + q, tap = col / COUT, co = col % COUT;
                    atomicAdd(a.dw + ((size_t)(ky0 * 3 + tap) * COUT + co) * CIN + ci, v[q]);
                }
            }
        }
    }
    if (do_bias && acc) atomicAdd(a.db + threadIdx.x % COUT, bsum);
    if (s_bad && threadIdx.x == 0) atomicExch(err, 1);
    asm volatile("cp.async.wait_all;" ::: "memory");
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
    __syncthreads();
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
    if (warp == 0)
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(TCOLS) : "memory");
}

template <int CIN, int COUT, int KYS>
static cudaError_t wgrad_tc_t(const WgradArgs &a, int sms, int *err, cudaStream_t s)
{
    typedef WgShape<CIN, COUT, KYS> S;
    const size_t smem = S::BYTES;
    cudaError_t e = cudaFuncSetAttribute(k_wgrad_tc<CIN, COUT, KYS>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         (int)smem);
    if (e != cudaSuccess) return e;
    constexpr int NKG = 3 / KYS;
    const long nunits = (long)a.B * (a.W / TC_TW) * ((a.H + WG_STRIP - 1) / WG_STRIP);
    long nsplit = sms / NKG > 0 ? sms / NKG : 1;   // about one block per SM
    if (nsplit > nunits) nsplit = nunits;
    k_wgrad_tc<CIN, COUT, KYS><<<(int)(NKG * nsplit), 128, smem, s>>>(a, err);
    return cudaGetLastError();
}

// the layers whose weight gradient takes tcgen05: c5 (96 -> 32, all nine taps
// in one block, 288 TMEM columns) and c4 (128 -> 64, a kernel row per block,
// 192 columns), rows of a multiple of 128 points
bool wgrad_tc_supported(int cin, int cout, int W)
{
    return W % TC_TW == 0 && ((cin == 96 && cout == 32) || (cin == 128 && cout == 64));
}

cudaError_t launch_wgrad_tc(int cin, int cout, const WgradArgs &a, int sms, int *err, cudaStream_t s)
{
    if (cin == 96 && cout == 32) return wgrad_tc_t<96, 32, 3>(a, sms, err, s);
    if (cin == 128 && cout == 64) return wgrad_tc_t<128, 64, 1>(a, sms, err, s);
    return cudaErrorInvalidValue;
}

} // namespace nn
