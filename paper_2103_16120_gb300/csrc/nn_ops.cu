// nn_ops.cu -- the memory-bound pieces of the learned preconditioner's network:
// 2x2 mean pooling, nearest-neighbour upsampling joined to a skip connection
// (channel concatenation), their adjoints with the ReLU derivative, the loss,
// the input packing, the parameter packing and the AdamW update.  All
// activations are NHWC BF16; sizes are those of the finer level.
#include <cuda_bf16.h>
#include <cstdint>

#include "nn_internal.h"

namespace nn {

static int blocks_for(size_t n, int threads)
{
    size_t b = (n + threads - 1) / threads;
    if (b > 152 * 16) b = 152 * 16;
    return b < 1 ? 1 : (int)b;
}

// ---------------------------------------------------------------------------
// y[b, h, w, c] = mean of x over the 2x2 block (2h.., 2w..)   (y is H/2 x W/2)
__global__ void k_pool(const __nv_bfloat162 *x, __nv_bfloat162 *y, int B, int H, int W, int C2)
{
    const int Ho = H / 2, Wo = W / 2;
    const size_t n = (size_t)B * Ho * Wo * C2;
    for (size_t q = blockIdx.x * (size_t)blockDim.x + threadIdx.x; q < n; q += (size_t)gridDim.x * blockDim.x) {
        const int c = (int)(q % C2);
        const size_t pix = q / C2;
        const int wo = (int)(pix % Wo), ho = (int)((pix / Wo) % Ho), b = (int)(pix / Wo / Ho);
        const size_t i00 = (((size_t)b * H + 2 * ho) * W + 2 * wo) * C2 + c;
        const float2 a0 = __bfloat1622float2(x[i00]), a1 = __bfloat1622float2(x[i00 + C2]);
        const float2 a2 = __bfloat1622float2(x[i00 + (size_t)W * C2]), a3 = __bfloat1622float2(x[i00 + (size_t)W * C2 + C2]);
        y[q] = __floats2bfloat162_rn(0.25f * ((a0.x + a1.x) + (a2.x + a3.x)), 0.25f * ((a0.y + a1.y) + (a2.y + a3.y)));
    }
}

// out[b, h, w, :] = [coarse[b, h/2, w/2, 0:cc], skip[b, h, w, 0:cs]]   (16-byte pieces)
__global__ void k_cat_up(const uint4 *coarse, int cc8, const uint4 *skip, int cs8, uint4 *out, int B, int H, int W)
{
    const int c8 = cc8 + cs8;
    const size_t n = (size_t)B * H * W * c8;
    for (size_t q = blockIdx.x * (size_t)blockDim.x + threadIdx.x; q < n; q += (size_t)gridDim.x * blockDim.x) {
        const int c = (int)(q % c8);
        const size_t pix = q / c8;
        const int w = (int)(pix % W), h = (int)((pix / W) % H), b = (int)(pix / W / H);
        if (c < cc8) out[q] = coarse[(((size_t)b * (H / 2) + h / 2) * (W / 2) + w / 2) * cc8 + c];
        else out[q] = skip[pix * cs8 + (c - cc8)];
    }
}

// adjoint of k_cat_up: gz_coarse = (sum over the 2x2 block of gcat[..., 0:cc]) * (a_coarse > 0)
__global__ void k_up_bwd(const float *gcat, int cc, int cs, const __nv_bfloat16 *a_coarse,
                         __nv_bfloat16 *gz, int B, int H, int W)
{
    const int Ho = H / 2, Wo = W / 2, ct = cc + cs;
    const size_t n = (size_t)B * Ho * Wo * cc;
    for (size_t q = blockIdx.x * (size_t)blockDim.x + threadIdx.x; q < n; q += (size_t)gridDim.x * blockDim.x) {
        const int c = (int)(q % cc);
        const size_t pix = q / cc;
        const int wo = (int)(pix % Wo), ho = (int)((pix / Wo) % Ho), b = (int)(pix / Wo / Ho);
        const size_t i00 = (((size_t)b * H + 2 * ho) * W + 2 * wo) * ct + c;
        const float s = (gcat[i00] + gcat[i00 + ct]) + (gcat[i00 + (size_t)W * ct] + gcat[i00 + (size_t)W * ct + ct]);
        gz[q] = __float2bfloat16_rn(__bfloat162float(a_coarse[q]) > 0.f ? s : 0.f);
    }
}

// the skip part of gcat, in FP32
__global__ void k_skip_bwd(const float *gcat, int cc, int cs, float *gskip, int B, int H, int W)
{
    const size_t n = (size_t)B * H * W * cs;
    for (size_t q = blockIdx.x * (size_t)blockDim.x + threadIdx.x; q < n; q += (size_t)gridDim.x * blockDim.x) {
        const size_t pix = q / cs;
        gskip[q] = gcat[pix * (cc + cs) + cc + (int)(q % cs)];
    }
}

// gz = (g_skip + pool-adjoint of g_pooled) * (a > 0)
__global__ void k_pool_bwd(const float *gskip, const float *gp, const __nv_bfloat16 *a, __nv_bfloat16 *gz,
                           int B, int H, int W, int C)
{
    const size_t n = (size_t)B * H * W * C;
    for (size_t q = blockIdx.x * (size_t)blockDim.x + threadIdx.x; q < n; q += (size_t)gridDim.x * blockDim.x) {
        const int c = (int)(q % C);
        const size_t pix = q / C;
        const int w = (int)(pix % W), h = (int)((pix / W) % H), b = (int)(pix / W / H);
        const float g = gskip[q] + 0.25f * gp[(((size_t)b * (H / 2) + h / 2) * (W / 2) + w / 2) * C + c];
        gz[q] = __float2bfloat16_rn(__bfloat162float(a[q]) > 0.f ? g : 0.f);
    }
}

// squared error, its gradient (padded to 16 BF16 channels) and the loss sum
__global__ void k_loss(const float *y, const float *t, __nv_bfloat16 *gy16, double *loss, size_t n)
{
    const double inv = 1.0 / (double)n;
    double part = 0.0;
    for (size_t q = blockIdx.x * (size_t)blockDim.x + threadIdx.x; q < n; q += (size_t)gridDim.x * blockDim.x) {
        const float d = y[q] - t[q];
        part += (double)d * d;
        uint4 *o = (uint4 *)(gy16 + q * 16);
        const __nv_bfloat16 g0 = __float2bfloat16_rn((float)(2.0 * inv) * d);
        uint4 first = make_uint4(0, 0, 0, 0);
        first.x = (unsigned)__bfloat16_as_ushort(g0);
        o[0] = first;
        o[1] = make_uint4(0, 0, 0, 0);
    }
    // block sum in a fixed order, one atomic per block
    __shared__ double red[32];
    for (int off = 16; off > 0; off >>= 1) part += __shfl_xor_sync(0xffffffffu, part, off);
    if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = part;
    __syncthreads();
    if (threadIdx.x == 0) {
        double s = 0.0;
        for (int w = 0; w < (int)(blockDim.x >> 5); ++w) s += red[w];
        atomicAdd(loss, s * inv);
    }
}

// x0 [B][4][H][W] FP32 -> [B][H][W][16] BF16 (channels 4..15 zero)
__global__ void k_pack_input(const float *x0, __nv_bfloat16 *xb, int B, int H, int W)
{
    const size_t hw = (size_t)H * W, n = (size_t)B * hw;
    for (size_t q = blockIdx.x * (size_t)blockDim.x + threadIdx.x; q < n; q += (size_t)gridDim.x * blockDim.x) {
        const size_t b = q / hw, p = q % hw;
        __nv_bfloat16 v[16];
#pragma unroll
        for (int c = 0; c < 16; ++c) v[c] = __float2bfloat16_rn(c < 4 ? x0[(b * 4 + c) * hw + p] : 0.f);
        uint4 *o = (uint4 *)(xb + q * 16);
        o[0] = *(const uint4 *)&v[0];
        o[1] = *(const uint4 *)&v[8];
    }
}

// ---------------------------------------------------------------------------
// parameters
// ---------------------------------------------------------------------------
size_t param_offset(int layer)
{
    size_t off = 0;
    for (int l = 0; l < layer; ++l) off += (size_t)LAYER[l].cout * LAYER[l].cin * 9 + LAYER[l].cout;
    return off;
}

size_t param_count() { return param_offset(NLAYERS); }

// layer offsets and shapes, passed by value to the kernels
struct LayerPtrs {
    int off[NLAYERS + 1];
    LayerShape sh[NLAYERS];
};

// forward weights wf[tap][o][c] = w[o][c][tap]; input-gradient weights
// wd[tap'][c][o] = w[o][c][8 - tap'] (taps flipped, channels swapped);
// padded channels are zero
__global__ void k_pack(PackArgs a, LayerPtrs lp)
{
    for (int l = 0; l < NLAYERS; ++l) {
        const LayerShape S = lp.sh[l];
        const float *w = a.master + lp.off[l];
        const int nf = 9 * S.cout_pad * S.cin_pad;
        for (int q = blockIdx.x * blockDim.x + threadIdx.x; q < nf; q += gridDim.x * blockDim.x) {
            // forward
            {
                const int c = q % S.cin_pad, o = (q / S.cin_pad) % S.cout_pad, tap = q / S.cin_pad / S.cout_pad;
                const float v = (c < S.cin && o < S.cout) ? w[(o * S.cin + c) * 9 + tap] : 0.f;
                a.wf[l][q] = __float2bfloat16_rn(v);
            }
            // input gradient: [tap'][c][o]
            {
                const int o = q % S.cout_pad, c = (q / S.cout_pad) % S.cin_pad, tp = q / S.cout_pad / S.cin_pad;
                const float v = (c < S.cin && o < S.cout) ? w[(o * S.cin + c) * 9 + (8 - tp)] : 0.f;
                a.wd[l][q] = __float2bfloat16_rn(v);
            }
        }
        for (int q = blockIdx.x * blockDim.x + threadIdx.x; q < S.cout_pad; q += gridDim.x * blockDim.x)
            a.bias[l][q] = q < S.cout ? w[S.cout * S.cin * 9 + q] : 0.f;
    }
}

__global__ void k_flatten_grad(GradPtrs g, LayerPtrs lp, float *flat)
{
    for (int l = 0; l < NLAYERS; ++l) {
        const LayerShape S = lp.sh[l];
        const int nw = S.cout * S.cin * 9;
        for (int q = blockIdx.x * blockDim.x + threadIdx.x; q < nw + S.cout; q += gridDim.x * blockDim.x) {
            float v;
            if (q < nw) {
                const int tap = q % 9, c = (q / 9) % S.cin, o = q / 9 / S.cin;
                v = g.dw[l][((size_t)tap * S.cout_pad + o) * S.cin_pad + c];
            } else {
                v = g.db[l][q - nw];
            }
            flat[lp.off[l] + q] = v;
        }
    }
}

// AdamW (decoupled weight decay on weights, none on biases)
__global__ void k_adamw(float *p, float *m, float *v, const float *g, size_t n, float lr, float b1, float b2,
                        float eps, float wd, float c1, float c2, LayerPtrs lp)
{
    for (size_t q = blockIdx.x * (size_t)blockDim.x + threadIdx.x; q < n; q += (size_t)gridDim.x * blockDim.x) {
        int l = 0;
        while (l + 1 < NLAYERS && (size_t)lp.off[l + 1] <= q) ++l;
        const bool bias = q >= (size_t)lp.off[l] + (size_t)lp.sh[l].cout * lp.sh[l].cin * 9;
        const float gq = g[q];
        const float mq = b1 * m[q] + (1.f - b1) * gq;
        const float vq = b2 * v[q] + (1.f - b2) * gq * gq;
        m[q] = mq;
        v[q] = vq;
        const float mh = mq / c1, vh = vq / c2;
        p[q] -= lr * (mh / (sqrtf(vh) + eps) + (bias ? 0.f : wd * p[q]));
    }
}

static LayerPtrs layer_ptrs()
{
    LayerPtrs lp;
    for (int l = 0; l <= NLAYERS; ++l) lp.off[l] = (int)param_offset(l);
    for (int l = 0; l < NLAYERS; ++l) lp.sh[l] = LAYER[l];
    return lp;
}

// ---------------------------------------------------------------------------
// launchers
// ---------------------------------------------------------------------------
cudaError_t launch_pool(const __nv_bfloat16 *x, __nv_bfloat16 *y, int B, int H, int W, int C, cudaStream_t s)
{
    const size_t n = (size_t)B * (H / 2) * (W / 2) * (C / 2);
    k_pool<<<blocks_for(n, 256), 256, 0, s>>>((const __nv_bfloat162 *)x, (__nv_bfloat162 *)y, B, H, W, C / 2);
    return cudaGetLastError();
}

cudaError_t launch_cat_up(const __nv_bfloat16 *coarse, int cc, const __nv_bfloat16 *skip, int cs,
                          __nv_bfloat16 *out, int B, int H, int W, cudaStream_t s)
{
    const size_t n = (size_t)B * H * W * ((cc + cs) / 8);
    k_cat_up<<<blocks_for(n, 256), 256, 0, s>>>((const uint4 *)coarse, cc / 8, (const uint4 *)skip, cs / 8,
                                                 (uint4 *)out, B, H, W);
    return cudaGetLastError();
}

cudaError_t launch_split_up_bwd(const float *gcat, int cc, int cs, const __nv_bfloat16 *a_coarse,
                                __nv_bfloat16 *gz_coarse, float *g_skip, int B, int H, int W, cudaStream_t s)
{
    const size_t n1 = (size_t)B * (H / 2) * (W / 2) * cc, n2 = (size_t)B * H * W * cs;
    k_up_bwd<<<blocks_for(n1, 256), 256, 0, s>>>(gcat, cc, cs, a_coarse, gz_coarse, B, H, W);
    k_skip_bwd<<<blocks_for(n2, 256), 256, 0, s>>>(gcat, cc, cs, g_skip, B, H, W);
    return cudaGetLastError();
}

cudaError_t launch_pool_bwd(const float *g_skip, const float *g_pooled, const __nv_bfloat16 *a,
                            __nv_bfloat16 *gz, int B, int H, int W, int C, cudaStream_t s)
{
    const size_t n = (size_t)B * H * W * C;
    k_pool_bwd<<<blocks_for(n, 256), 256, 0, s>>>(g_skip, g_pooled, a, gz, B, H, W, C);
    return cudaGetLastError();
}

cudaError_t launch_loss(const float *y, const float *target, __nv_bfloat16 *gy16, double *loss, int B, int H, int W,
                        cudaStream_t s)
{
    const size_t n = (size_t)B * H * W;
    k_loss<<<blocks_for(n, 256), 256, 0, s>>>(y, target, gy16, loss, n);
    return cudaGetLastError();
}

cudaError_t launch_pack_input(const float *x0, __nv_bfloat16 *xb, int B, int H, int W, cudaStream_t s)
{
    const size_t n = (size_t)B * H * W;
    k_pack_input<<<blocks_for(n, 256), 256, 0, s>>>(x0, xb, B, H, W);
    return cudaGetLastError();
}

cudaError_t launch_pack(const PackArgs &a, cudaStream_t s)
{
    k_pack<<<64, 256, 0, s>>>(a, layer_ptrs());
    return cudaGetLastError();
}

cudaError_t launch_flatten_grad(const GradPtrs &g, float *flat, cudaStream_t s)
{
    k_flatten_grad<<<64, 256, 0, s>>>(g, layer_ptrs(), flat);
    return cudaGetLastError();
}

cudaError_t launch_adamw(float *master, float *m, float *v, const float *flat_grad, size_t n, float lr, float beta1,
                         float beta2, float eps, float wd, int t, cudaStream_t s)
{
    const float c1 = 1.f - powf(beta1, (float)t), c2 = 1.f - powf(beta2, (float)t);
    k_adamw<<<blocks_for(n, 256), 256, 0, s>>>(master, m, v, flat_grad, n, lr, beta1, beta2, eps, wd, c1, c2,
                                               layer_ptrs());
    return cudaGetLastError();
}

} // namespace nn
