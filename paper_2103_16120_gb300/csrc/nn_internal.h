// nn_internal.h -- host-side interfaces of the learned preconditioner's
// kernels (nn_conv.cu, nn_ops.cu) used by the model driver (nn_model.cu).
#pragma once

#include <cuda_bf16.h>
#include <cuda_runtime.h>
#include <stddef.h>

namespace nn {

// Resident blocks per SM of kernel KERN for a block size and a dynamic
// shared-memory size, asked of the runtime once per (device, size) and kept,
// with the kernel's shared-memory limit raised as needed (it only grows).
// The network then launches the same way while a stream is being captured
// into a graph (the learned preconditioner's device-side loop), where the
// occupancy query may not run, and a launch recorded in a graph keeps a
// limit large enough.
template <auto KERN>
inline cudaError_t occupancy_once(int threads, size_t smem, int *bps)
{
    struct Entry { int dev, threads; size_t smem; int bps; };
    static Entry seen[16];
    static int n = 0;
    static size_t limit[8] = {};
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return e;
    for (int q = 0; q < n; ++q)
        if (seen[q].dev == dev && seen[q].threads == threads && seen[q].smem == smem) {
            *bps = seen[q].bps;
            return cudaSuccess;
        }
    size_t &lim = limit[dev & 7];
    if (smem > lim) {
        e = cudaFuncSetAttribute(KERN, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        if (e != cudaSuccess) return e;
        lim = smem;
    }
    e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(bps, KERN, threads, smem);
    if (e != cudaSuccess) return e;
    if (n < 16) seen[n++] = Entry{dev, threads, smem, *bps};
    return cudaSuccess;
}

// 3x3 convolution over NHWC BF16 activations (see nn_conv.cu)
struct ConvArgs {
    const __nv_bfloat16 *x;     // [B][H][W][cin]
    const __nv_bfloat16 *w;     // [9][cout][cin]
    const float *bias;          // [cout] or null
    __nv_bfloat16 *y;           // [B][H][W][cout] (unless yf is set)
    float *yf;                  // FP32 output [B][H][W][yf_c] of channels < yf_c, or null
    int yf_c;
    const __nv_bfloat16 *mask;  // [B][H][W][cout]: zero the output where mask <= 0 (ReLU derivative), or null
    int B, H, W;
    int relu;
};

struct WgradArgs {
    const __nv_bfloat16 *g;     // [B][H][W][cout]  gradient at the layer output (pre-activation)
    const __nv_bfloat16 *x;     // [B][H][W][cin]   layer input
    float *dw;                  // [9][cout][cin]   accumulated (FP32)
    float *db;                  // [cout] accumulated, or null
    int B, H, W;
};

cudaError_t launch_conv(int cin, int cout, bool dgrad, const ConvArgs &a, int sms, cudaStream_t s);
// the same convolution on tcgen05 (nn_tc.cu) where its rows are a multiple of
// 128 points and the operands fit in shared memory; err (device) is set if a
// tensor-core wait ran out
bool conv_tc_supported(int cin, int cout, bool dgrad, int W);
cudaError_t launch_conv_tc(int cin, int cout, bool dgrad, const ConvArgs &a, int sms, int *err, cudaStream_t s);
inline cudaError_t launch_conv_auto(int cin, int cout, bool dgrad, const ConvArgs &a, int sms, int *err,
                                    cudaStream_t s)
{
    return conv_tc_supported(cin, cout, dgrad, a.W) ? launch_conv_tc(cin, cout, dgrad, a, sms, err, s)
                                                    : launch_conv(cin, cout, dgrad, a, sms, s);
}
cudaError_t launch_wgrad(int cin, int cout, const WgradArgs &a, int sms, cudaStream_t s);
// the weight gradient on tcgen05 (nn_tc.cu) for the layers it takes
bool wgrad_tc_supported(int cin, int cout, int W);
cudaError_t launch_wgrad_tc(int cin, int cout, const WgradArgs &a, int sms, int *err, cudaStream_t s);
inline cudaError_t launch_wgrad_auto(int cin, int cout, const WgradArgs &a, int sms, int *err, cudaStream_t s)
{
    return wgrad_tc_supported(cin, cout, a.W) ? launch_wgrad_tc(cin, cout, a, sms, err, s)
                                              : launch_wgrad(cin, cout, a, sms, s);
}

// elementwise and small kernels (nn_ops.cu); shapes are of the fine level
cudaError_t launch_pool(const __nv_bfloat16 *x, __nv_bfloat16 *y, int B, int H, int W, int C, cudaStream_t s);
cudaError_t launch_cat_up(const __nv_bfloat16 *coarse, int cc, const __nv_bfloat16 *skip, int cs,
                          __nv_bfloat16 *out, int B, int H, int W, cudaStream_t s);
cudaError_t launch_split_up_bwd(const float *gcat, int cc, int cs, const __nv_bfloat16 *a_coarse,
                                __nv_bfloat16 *gz_coarse, float *g_skip, int B, int H, int W, cudaStream_t s);
cudaError_t launch_pool_bwd(const float *g_skip, const float *g_pooled, const __nv_bfloat16 *a,
                            __nv_bfloat16 *gz, int B, int H, int W, int C, cudaStream_t s);
// gy16[p][0] = 2 (y - target) / (B H W), gy16[p][1..15] = 0; loss += sum (y - target)^2 / (B H W)
cudaError_t launch_loss(const float *y, const float *target, __nv_bfloat16 *gy16, double *loss, int B, int H, int W,
                        cudaStream_t s);
cudaError_t launch_pack_input(const float *x0, __nv_bfloat16 *xb, int B, int H, int W, cudaStream_t s);

// parameters: flat FP32 vector in the order [layer][w: cout][cin][3][3], [layer][b]
constexpr int NLAYERS = 6;
struct LayerShape {
    int cin, cout, cin_pad, cout_pad, level;   // channels, as stored on the GPU, resolution level
};
constexpr LayerShape LAYER[NLAYERS] = {{4, 32, 16, 32, 0},  {32, 64, 32, 64, 1}, {64, 64, 64, 64, 2},
                                       {128, 64, 128, 64, 1}, {96, 32, 96, 32, 0}, {32, 1, 32, 16, 0}};
size_t param_count();
size_t param_offset(int layer);   // start of layer's w in the flat vector (b follows w)

struct PackArgs {
    const float *master;                        // flat FP32 parameters
    __nv_bfloat16 *wf[NLAYERS];                 // forward weights [9][cout_pad][cin_pad]
    __nv_bfloat16 *wd[NLAYERS];                 // input-gradient weights [9][cin_pad][cout_pad], taps flipped
    float *bias[NLAYERS];                       // [cout_pad]
};
cudaError_t launch_pack(const PackArgs &a, cudaStream_t s);

struct GradPtrs {
    const float *dw[NLAYERS];                   // [9][cout_pad][cin_pad]
    const float *db[NLAYERS];                   // [cout_pad]
};
// flat gradient (oracle order) from the kernel-native gradient buffers
cudaError_t launch_flatten_grad(const GradPtrs &g, float *flat, cudaStream_t s);
cudaError_t launch_adamw(float *master, float *m, float *v, const float *flat_grad, size_t n, float lr, float beta1,
                         float beta2, float eps, float wd, int t, cudaStream_t s);

} // namespace nn
