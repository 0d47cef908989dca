// nn_conv.cu -- 3x3 convolutions of the learned preconditioner on the tensor
// cores (BF16 operands, FP32 accumulation, mma.sync m16n8k16), as implicit
// GEMMs over NHWC activations [B][H][W][C]:
//
//   k_conv   y[p][o] = b[o] + sum_{tap, c} w[tap][o][c] xt[p + tap][c]
//            (forward: xt is x with the sphere halo -- periodic longitude,
//            across-pole ghost rows; DGRAD: the adjoint of that halo, i.e.
//            zero rows beyond the poles plus, on a pole row, the extra taps
//            that collect what the ghost row had copied from it)
//   k_wgrad  dw[tap][o][c] += sum_p g[p][o] xt[p + tap][c]   (split over pixels)
//
// The tap order is ky * 3 + kx with (ky, kx) = (1, 1) the centre; the weight
// rows are [tap][o][c] with c contiguous.  A block works on tiles of TW = 64
// (or W, when W < 64) consecutive points of one latitude row: it stages the
// tile's three input rows with their halo in shared memory once (cp.async)
// and feeds the nine taps to the tensor cores with ldmatrix row addresses
// shifted by the tap -- no im2col buffer.
#include <cuda_bf16.h>
#include <cstdint>

#include "nn_internal.h"

namespace nn {

__device__ __forceinline__ unsigned smem_u32(const void *p) { return (unsigned)__cvta_generic_to_shared(p); }

__device__ __forceinline__ void cp16(void *s, const void *g)
{
    asm volatile("cp.async.cg.shared.global [%0], [%1], 16;" ::"r"(smem_u32(s)), "l"(g) : "memory");
}
__device__ __forceinline__ void cp_wait() { asm volatile("cp.async.wait_all;" ::: "memory"); }

__device__ __forceinline__ void ldsm_x4(unsigned (&r)[4], const void *p)
{
    asm volatile("ldmatrix.sync.aligned.m8n8.x4.shared.b16 {%0,%1,%2,%3}, [%4];"
                 : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]) : "r"(smem_u32(p)));
}
__device__ __forceinline__ void ldsm_x4_t(unsigned (&r)[4], const void *p)
{
    asm volatile("ldmatrix.sync.aligned.m8n8.x4.trans.shared.b16 {%0,%1,%2,%3}, [%4];"
                 : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]) : "r"(smem_u32(p)));
}

// D += A (16x16, row) * B (16x8, col), BF16 in, FP32 accumulate
__device__ __forceinline__ void mma16816(float (&d)[4], const unsigned (&a)[4], unsigned b0, unsigned b1)
{
    asm volatile("mma.sync.aligned.m16n8k16.row.col.f32.bf16.bf16.f32 "
                 "{%0,%1,%2,%3}, {%4,%5,%6,%7}, {%8,%9}, {%0,%1,%2,%3};"
                 : "+f"(d[0]), "+f"(d[1]), "+f"(d[2]), "+f"(d[3])
                 : "r"(a[0]), "r"(a[1]), "r"(a[2]), "r"(a[3]), "r"(b0), "r"(b1));
}

// shared-memory row pitch (elements) of a C-channel pixel: 8 extra elements
// (16 bytes) put the eight rows an ldmatrix reads on distinct bank groups
__host__ __device__ constexpr int pitch(int c) { return c + 8; }

// ---------------------------------------------------------------------------
// forward / input-gradient convolution
// ---------------------------------------------------------------------------
template <int CIN, int COUT, bool DGRAD>
__global__ void __launch_bounds__(128) k_conv(ConvArgs a)
{
    constexpr int NT = COUT / 8;             // n-tiles of 8 output channels
    constexpr int KS = CIN / 16;             // k-steps of 16 input channels per tap
    constexpr int PI = pitch(CIN);
    extern __shared__ __align__(16) unsigned char smem[];
    __nv_bfloat16 *Ws = (__nv_bfloat16 *)smem;                       // [9][COUT][PI]
    __nv_bfloat16 *Xs = Ws + 9 * COUT * PI;                          // [4][TW + 2][PI]
    const int H = a.H, W = a.W, TW = W < 64 ? W : 64;
    const int nseg = W / TW;
    const long ntiles = (long)a.B * H * nseg;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;

    // weights, once per block
    for (int q = threadIdx.x; q < 9 * COUT * (CIN / 8); q += blockDim.x) {
        const int row = q / (CIN / 8), ch = q % (CIN / 8);
        cp16(Ws + row * PI + ch * 8, a.w + (size_t)row * CIN + ch * 8);
    }

    for (long tile = blockIdx.x; tile < ntiles; tile += gridDim.x) {
        const int seg = (int)(tile % nseg);
        const long bh = tile / nseg;
        const int h = (int)(bh % H), b = (int)(bh / H);
        const int w0 = seg * TW;
        const bool pole = DGRAD && (h == 0 || h == H - 1);
        const int nrows = pole ? 4 : 3;
        __syncthreads();                         // previous tile's reads are done
        // stage rows h-1, h, h+1 (and, for DGRAD on a pole row, the pole row
        // shifted by half a circle) with one point of halo on each side
        for (int q = threadIdx.x; q < nrows * (TW + 2) * (CIN / 8); q += blockDim.x) {
            const int ch = q % (CIN / 8);
            const int cpt = (q / (CIN / 8)) % (TW + 2);
            const int r = q / (CIN / 8) / (TW + 2);
            int hs, shift = 0;
            bool zero = false;
            if (r < 3) {
                hs = h - 1 + r;
                if (hs < 0 || hs >= H) {
                    if (DGRAD) zero = true;
                    else { hs = hs < 0 ? 0 : H - 1; shift = W / 2; }
                }
            } else {
                hs = h; shift = W / 2;
            }
            __nv_bfloat16 *dst = Xs + (r * (TW + 2) + cpt) * PI + ch * 8;
            if (zero) {
                *(uint4 *)dst = make_uint4(0, 0, 0, 0);
            } else {
                int ws = w0 - 1 + cpt + shift;
                ws %= W;
                if (ws < 0) ws += W;
                cp16(dst, a.x + (((size_t)b * H + hs) * W + ws) * CIN + ch * 8);
            }
        }
        cp_wait();
        __syncthreads();

        const int p0 = warp * 16;
        if (p0 < TW) {
            float acc[NT][4];
#pragma unroll
            for (int j = 0; j < NT; ++j) acc[j][0] = acc[j][1] = acc[j][2] = acc[j][3] = 0.f;
            const int arow = p0 + (lane & 7) + 8 * ((lane >> 3) & 1);     // A row (point) of this lane
            const int akof = 8 * (lane >> 4);                             // A k offset
            const int brow = (lane & 7) + 8 * (lane >> 4);                // B row (out channel) in a pair
            const int bkof = 8 * ((lane >> 3) & 1);                       // B k offset
            // DGRAD pole row: the extra taps use weight row ky = 2 (row 0) or 0 (row H-1)
            const int ntap = pole ? 12 : 9;
            for (int t = 0; t < ntap; ++t) {
                int tap, xr;
                if (t < 9) { tap = t; xr = t / 3; }
                else { tap = (h == 0 ? 6 : 0) + (t - 9); xr = 3; }
                const int kx = tap % 3;
                const __nv_bfloat16 *xa = Xs + (xr * (TW + 2) + arow + kx) * PI + akof;
                const __nv_bfloat16 *wb = Ws + (tap * COUT + brow) * PI + bkof;
#pragma unroll
                for (int ks = 0; ks < KS; ++ks) {
                    unsigned af[4];
                    ldsm_x4(af, xa + ks * 16);
#pragma unroll
                    for (int jp = 0; jp < NT / 2; ++jp) {
                        unsigned bf[4];
                        ldsm_x4(bf, wb + jp * 16 * PI + ks * 16);
                        mma16816(acc[2 * jp], af, bf[0], bf[1]);
                        mma16816(acc[2 * jp + 1], af, bf[2], bf[3]);
                    }
                }
            }
            // epilogue: bias, ReLU or mask, store of the 16 points x COUT
            const int g = lane >> 2, tg = lane & 3;
            const size_t pix = ((size_t)b * H + h) * W + w0 + p0;      // first point of the warp
#pragma unroll
            for (int j = 0; j < NT; ++j) {
                const int co = 8 * j + 2 * tg;
                const float b0 = a.bias ? a.bias[co] : 0.f, b1 = a.bias ? a.bias[co + 1] : 0.f;
                float v[4] = {acc[j][0] + b0, acc[j][1] + b1, acc[j][2] + b0, acc[j][3] + b1};
                if (a.relu)
#pragma unroll
                    for (int q = 0; q < 4; ++q) v[q] = fmaxf(v[q], 0.f);
                if (a.mask) {
#pragma unroll
                    for (int q = 0; q < 4; ++q) {
                        const size_t idx = (pix + g + 8 * (q >> 1)) * COUT + co + (q & 1);
                        if (!(__bfloat162float(a.mask[idx]) > 0.f)) v[q] = 0.f;
                    }
                }
                if (a.yf) {
#pragma unroll
                    for (int q = 0; q < 4; ++q) {
                        const int c = co + (q & 1);
                        if (c < a.yf_c) a.yf[(pix + g + 8 * (q >> 1)) * a.yf_c + c] = v[q];
                    }
                } else {
                    *(__nv_bfloat162 *)(a.y + (pix + g) * COUT + co) = __floats2bfloat162_rn(v[0], v[1]);
                    *(__nv_bfloat162 *)(a.y + (pix + g + 8) * COUT + co) = __floats2bfloat162_rn(v[2], v[3]);
                }
            }
        }
    }
}

// ---------------------------------------------------------------------------
// weight gradient: block (ky, c-block, split) accumulates the three taps of
// kernel row ky for COUT x NCI weights over its share of the tiles
// ---------------------------------------------------------------------------
template <int CIN, int COUT, int NCI>
__global__ void __launch_bounds__(COUT * 2) k_wgrad(WgradArgs a)
{
    constexpr int NTJ = NCI / 8;                 // n-tiles (input channels)
    constexpr int PG = pitch(COUT), PX = pitch(NCI);
    extern __shared__ __align__(16) unsigned char smem[];
    const int H = a.H, W = a.W, TW = W < 64 ? W : 64;
    __nv_bfloat16 *Gs = (__nv_bfloat16 *)smem;                       // [TW][PG]
    __nv_bfloat16 *Xs = Gs + 64 * PG;                                // [TW + 2][PX]
    const int ky = blockIdx.x % 3;
    const int cb = (blockIdx.x / 3) % (CIN / NCI);
    const int split = blockIdx.x / 3 / (CIN / NCI);
    const int nsplit = gridDim.x / 3 / (CIN / NCI);
    const int nseg = W / TW;
    const long ntiles = (long)a.B * H * nseg;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const bool do_bias = a.db && ky == 0 && cb == 0;

    float acc[3][NTJ][4];
#pragma unroll
    for (int kx = 0; kx < 3; ++kx)
#pragma unroll
        for (int j = 0; j < NTJ; ++j) acc[kx][j][0] = acc[kx][j][1] = acc[kx][j][2] = acc[kx][j][3] = 0.f;
    float bsum = 0.f;

    for (long tile = split; tile < ntiles; tile += nsplit) {
        const int seg = (int)(tile % nseg);
        const long bh = tile / nseg;
        const int h = (int)(bh % H), b = (int)(bh / H);
        const int w0 = seg * TW;
        __syncthreads();
        // gradient tile [TW][COUT]
        const __nv_bfloat16 *gsrc = a.g + (((size_t)b * H + h) * W + w0) * COUT;
        for (int q = threadIdx.x; q < TW * (COUT / 8); q += blockDim.x) {
            const int p = q / (COUT / 8), ch = q % (COUT / 8);
            cp16(Gs + p * PG + ch * 8, gsrc + (size_t)p * COUT + ch * 8);
        }
        // input row h + ky - 1 with the sphere halo, channels cb*NCI ..
        int hs = h - 1 + ky, shift = 0;
        if (hs < 0) { hs = 0; shift = W / 2; }
        else if (hs >= H) { hs = H - 1; shift = W / 2; }
        for (int q = threadIdx.x; q < (TW + 2) * (NCI / 8); q += blockDim.x) {
            const int cpt = q / (NCI / 8), ch = q % (NCI / 8);
            int ws = (w0 - 1 + cpt + shift) % W;
            if (ws < 0) ws += W;
            cp16(Xs + cpt * PX + ch * 8, a.x + (((size_t)b * H + hs) * W + ws) * CIN + cb * NCI + ch * 8);
        }
        cp_wait();
        __syncthreads();
        if (do_bias && threadIdx.x < COUT)
            for (int p = 0; p < TW; ++p) bsum += __bfloat162float(Gs[p * PG + threadIdx.x]);
        // A = g^T (16 out channels of this warp x 16 points), B = xt (16 points x 8 channels)
        const int m = lane >> 3, r8 = lane & 7;
        for (int k0 = 0; k0 < TW; k0 += 16) {
            unsigned af[4];
            ldsm_x4_t(af, Gs + (k0 + 8 * (m >> 1) + r8) * PG + warp * 16 + 8 * (m & 1));
#pragma unroll
            for (int kx = 0; kx < 3; ++kx) {
#pragma unroll
                for (int jp = 0; jp < NTJ / 2; ++jp) {
                    unsigned bf[4];
                    ldsm_x4_t(bf, Xs + (k0 + kx + 8 * (m & 1) + r8) * PX + jp * 16 + 8 * (m >> 1));
                    mma16816(acc[kx][2 * jp], af, bf[0], bf[1]);
                    mma16816(acc[kx][2 * jp + 1], af, bf[2], bf[3]);
                }
            }
        }
    }
    // accumulate into dw[tap][o][c] (FP32)
    const int g = lane >> 2, tg = lane & 3;
#pragma unroll
    for (int kx = 0; kx < 3; ++kx) {
        float *dw = a.dw + (size_t)(ky * 3 + kx) * COUT * CIN;
#pragma unroll
        for (int j = 0; j < NTJ; ++j) {
            const int c = cb * NCI + 8 * j + 2 * tg;
            const int o = warp * 16 + g;
            atomicAdd(dw + (size_t)o * CIN + c, acc[kx][j][0]);
            atomicAdd(dw + (size_t)o * CIN + c + 1, acc[kx][j][1]);
            atomicAdd(dw + (size_t)(o + 8) * CIN + c, acc[kx][j][2]);
            atomicAdd(dw + (size_t)(o + 8) * CIN + c + 1, acc[kx][j][3]);
        }
    }
    if (do_bias && threadIdx.x < COUT) atomicAdd(a.db + threadIdx.x, bsum);
}

// ---------------------------------------------------------------------------
// host launchers
// ---------------------------------------------------------------------------
template <int CIN, int COUT, bool DGRAD>
static cudaError_t conv_t(const ConvArgs &a, int sms, cudaStream_t s)
{
    const int TW = a.W < 64 ? a.W : 64;
    const size_t smem = (size_t)(9 * COUT + (DGRAD ? 4 : 3) * (TW + 2)) * pitch(CIN) * 2;
    int bps = 0;
    cudaError_t e = occupancy_once<k_conv<CIN, COUT, DGRAD>>(128, smem, &bps);
    if (e != cudaSuccess) return e;
    if (bps < 1) return cudaErrorInvalidConfiguration;
    const long ntiles = (long)a.B * a.H * (a.W / TW);
    long grid = (long)bps * sms;
    if (grid > ntiles) grid = ntiles;
    k_conv<CIN, COUT, DGRAD><<<(int)grid, 128, smem, s>>>(a);
    return cudaGetLastError();
}

template <int CIN, int COUT, int NCI>
static cudaError_t wgrad_t(const WgradArgs &a, int sms, cudaStream_t s)
{
    const size_t smem = (size_t)(64 * pitch(COUT) + 66 * pitch(NCI)) * 2;
    cudaError_t e = cudaFuncSetAttribute(k_wgrad<CIN, COUT, NCI>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         (int)smem);
    if (e != cudaSuccess) return e;
    const int TW = a.W < 64 ? a.W : 64;
    const long ntiles = (long)a.B * a.H * (a.W / TW);
    const int per = 3 * (CIN / NCI);
    long nsplit = (4L * sms + per - 1) / per;
    if (nsplit > ntiles) nsplit = ntiles;
    if (nsplit < 1) nsplit = 1;
    k_wgrad<CIN, COUT, NCI><<<(int)(per * nsplit), COUT * 2, smem, s>>>(a);
    return cudaGetLastError();
}

cudaError_t launch_conv(int cin, int cout, bool dgrad, const ConvArgs &a, int sms, cudaStream_t s)
{
#define NN_CONV(CI, CO)                                                              \
    if (cin == CI && cout == CO)                                                     \
        return dgrad ? conv_t<CI, CO, true>(a, sms, s) : conv_t<CI, CO, false>(a, sms, s);
    NN_CONV(16, 32)   // c1 forward (4 inputs padded to 16); c6 input gradient (16 -> 32)
    NN_CONV(32, 64)   // c2 forward
    NN_CONV(64, 64)   // c3 forward and input gradient
    NN_CONV(128, 64)  // c4 forward
    NN_CONV(96, 32)   // c5 forward
    NN_CONV(32, 16)   // c6 forward (1 output padded to 16)
    NN_CONV(64, 32)   // c2 input gradient (64 -> 32)
    NN_CONV(64, 128)  // c4 input gradient (64 -> 128)
    NN_CONV(32, 96)   // c5 input gradient (32 -> 96)
#undef NN_CONV
    return cudaErrorInvalidValue;
}

cudaError_t launch_wgrad(int cin, int cout, const WgradArgs &a, int sms, cudaStream_t s)
{
    if (cin == 16 && cout == 32) return wgrad_t<16, 32, 16>(a, sms, s);
    if (cin == 32 && cout == 64) return wgrad_t<32, 64, 32>(a, sms, s);
    if (cin == 64 && cout == 64) return wgrad_t<64, 64, 64>(a, sms, s);
    if (cin == 128 && cout == 64) return wgrad_t<128, 64, 64>(a, sms, s);
    if (cin == 96 && cout == 32) return wgrad_t<96, 32, 32>(a, sms, s);
    if (cin == 32 && cout == 16) return wgrad_t<32, 16, 32>(a, sms, s);
    return cudaErrorInvalidValue;
}

} // namespace nn
