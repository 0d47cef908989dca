// nn_model.cu -- the learned preconditioner's model: parameters, activation
// buffers, forward and backward passes (tensor-core convolutions of
// nn_conv.cu, memory-bound pieces of nn_ops.cu), AdamW training steps, the
// network's inputs from a grid and the preconditioner e = s y / d; and the C
// ABI of include/sw_elliptic.h for all of it.
#include <cmath>
#include <cstring>
#include <new>
#include <string>

#include "../../include/sw_elliptic.h"
#include "nn_internal.h"
#include "sw_internal.h"

using namespace nn;

#define NCK(call)                                                                       \
    do {                                                                                \
        cudaError_t e_ = (call);                                                        \
        if (e_ != cudaSuccess)                                                          \
            return sw::api_fail(e_ == cudaErrorMemoryAllocation ? SW_ERR_OOM : SW_ERR_CUDA, \
                                (std::string(#call) + ": " + cudaGetErrorString(e_)).c_str()); \
    } while (0)

namespace {

typedef __nv_bfloat16 bf16;

struct Acts {
    size_t cap_n0 = 0, cap_hw = 0;   // capacity: points of a batch, points of one sample
    void *mem = nullptr;
    bf16 *x0b, *a1, *p1, *a2, *p2, *a3, *cat4, *a4, *cat5, *a5;
    float *y;
    bf16 *gy16, *gz5, *gz4, *gz3, *gz2, *gz1;
    float *gcat5, *gcat4, *gp2, *gp1;    // input gradients of the convolutions, FP32
    float *gskip1, *gskip2;
    float *x0f;                  // one sample's FP32 inputs (sw_model_apply)
    float *ef;                   // one sample's preconditioner output (solver)
    double *scal;                // [0]: sum r^2 (apply), [1]: loss
};

} // namespace

struct sw_model_s {
    int device = 0, sms = 0;
    size_t np = 0;
    void *pmem = nullptr;
    float *master, *m, *v, *gflat;
    bf16 *wf[NLAYERS], *wd[NLAYERS];
    float *bias[NLAYERS], *dw[NLAYERS], *db[NLAYERS];
    int *err;                    // device: a tensor-core wait ran out
    int t = 0;
    Acts A;
    // a number no other model or activation storage of this process has had:
    // a new one at creation and at every reallocation of the activations
    unsigned long long gen = 0;
};

static unsigned long long next_model_gen()
{
    static unsigned long long n = 0;
    return ++n;
}

namespace {

size_t al256(size_t x) { return (x + 255) & ~(size_t)255; }

sw_status check_shape(int B, int H, int W)
{
    if (B < 1) return sw::api_fail(SW_ERR_INVALID_ARG, "batch must be >= 1");
    if (H < 8 || (H & 3)) return sw::api_fail(SW_ERR_INVALID_ARG, "ny must be a multiple of 4 and >= 8");
    // every level's row splits into tiles of 64 points, or is one tile of a
    // multiple of 16 points
    for (int l = 0; l < 3; ++l) {
        const int Wl = W >> l;
        if ((W & ((1 << l) - 1)) || (Wl <= 64 ? (Wl & 15) : (Wl & 63)))
            return sw::api_fail(SW_ERR_INVALID_ARG, "nx must be 64, 128 or a multiple of 256");
    }
    return SW_OK;
}

// activation and gradient buffers for B samples of H x W (grown on demand)
sw_status ensure_acts(sw_model_s *M, int B, int H, int W)
{
    Acts &A = M->A;
    if (A.mem && A.cap_n0 >= (size_t)B * H * W && A.cap_hw >= (size_t)H * W) return SW_OK;
    if (A.mem) { cudaFree(A.mem); A.mem = nullptr; }
    M->gen = next_model_gen();
    const size_t N0 = (size_t)B * H * W, N1 = N0 / 4, N2 = N0 / 16;
    const size_t hb[] = {N0 * 16, N0 * 32, N1 * 32, N1 * 64, N2 * 64, N2 * 64, N1 * 128, N1 * 64, N0 * 96, N0 * 32,
                         N0 * 16, N0 * 32, N1 * 64, N2 * 64, N1 * 64, N0 * 32};
    const size_t hf[] = {N0 * 96, N1 * 128, N2 * 64, N1 * 32};
    size_t bytes = 0;
    for (size_t h : hb) bytes += al256(h * 2);
    for (size_t h : hf) bytes += al256(h * 4);
    bytes += al256(N0 * 4) + al256(N0 * 32 * 4) + al256(N1 * 64 * 4) + al256((size_t)4 * H * W * 4) +
             al256((size_t)H * W * 4) + al256(64);
    NCK(cudaMalloc(&A.mem, bytes));
    char *p = (char *)A.mem;
    bf16 **slots[] = {&A.x0b, &A.a1, &A.p1, &A.a2, &A.p2, &A.a3, &A.cat4, &A.a4, &A.cat5, &A.a5,
                      &A.gy16, &A.gz5, &A.gz4, &A.gz3, &A.gz2, &A.gz1};
    for (int q = 0; q < 16; ++q) { *slots[q] = (bf16 *)p; p += al256(hb[q] * 2); }
    float **fslots[] = {&A.gcat5, &A.gcat4, &A.gp2, &A.gp1};
    for (int q = 0; q < 4; ++q) { *fslots[q] = (float *)p; p += al256(hf[q] * 4); }
    A.y = (float *)p; p += al256(N0 * 4);
    A.gskip1 = (float *)p; p += al256(N0 * 32 * 4);
    A.gskip2 = (float *)p; p += al256(N1 * 64 * 4);
    A.x0f = (float *)p; p += al256((size_t)4 * H * W * 4);
    A.ef = (float *)p; p += al256((size_t)H * W * 4);
    A.scal = (double *)p;
    A.cap_n0 = N0;
    A.cap_hw = (size_t)H * W;
    return SW_OK;
}

sw_status check_err(sw_model_s *M)
{
    int e = 0;
    NCK(cudaMemcpy(&e, M->err, sizeof(int), cudaMemcpyDeviceToHost));
    if (e) return sw::api_fail(SW_ERR_TIMEOUT, "a tensor-core wait of the network ran out");
    return SW_OK;
}

ConvArgs conv_args(const bf16 *x, const bf16 *w, const float *bias, bf16 *y, int B, int H, int W, int relu)
{
    ConvArgs a;
    a.x = x; a.w = w; a.bias = bias; a.y = y; a.yf = nullptr; a.yf_c = 0; a.mask = nullptr;
    a.B = B; a.H = H; a.W = W; a.relu = relu;
    return a;
}

// an input-gradient convolution with FP32 output (rounded to BF16 once, by
// the consumer that feeds the next tensor-core operation)
ConvArgs dgrad_args(const bf16 *g, const bf16 *w, float *out, int cout, int B, int H, int W)
{
    ConvArgs a = conv_args(g, w, nullptr, nullptr, B, H, W, 0);
    a.yf = out;
    a.yf_c = cout;
    return a;
}

sw_status forward(sw_model_s *M, int B, int H, int W, const float *x0, cudaStream_t s)
{
    Acts &A = M->A;
    const int H1 = H / 2, W1 = W / 2, H2 = H / 4, W2 = W / 4;
    NCK(launch_pack_input(x0, A.x0b, B, H, W, s));
    NCK(launch_conv_auto(16, 32, false, conv_args(A.x0b, M->wf[0], M->bias[0], A.a1, B, H, W, 1), M->sms, M->err, s));
    NCK(launch_pool(A.a1, A.p1, B, H, W, 32, s));
    NCK(launch_conv_auto(32, 64, false, conv_args(A.p1, M->wf[1], M->bias[1], A.a2, B, H1, W1, 1), M->sms, M->err, s));
    NCK(launch_pool(A.a2, A.p2, B, H1, W1, 64, s));
    NCK(launch_conv_auto(64, 64, false, conv_args(A.p2, M->wf[2], M->bias[2], A.a3, B, H2, W2, 1), M->sms, M->err, s));
    NCK(launch_cat_up(A.a3, 64, A.a2, 64, A.cat4, B, H1, W1, s));
    NCK(launch_conv_auto(128, 64, false, conv_args(A.cat4, M->wf[3], M->bias[3], A.a4, B, H1, W1, 1), M->sms, M->err, s));
    NCK(launch_cat_up(A.a4, 64, A.a1, 32, A.cat5, B, H, W, s));
    NCK(launch_conv_auto(96, 32, false, conv_args(A.cat5, M->wf[4], M->bias[4], A.a5, B, H, W, 1), M->sms, M->err, s));
    ConvArgs o = conv_args(A.a5, M->wf[5], M->bias[5], nullptr, B, H, W, 0);
    o.yf = A.y; o.yf_c = 1;
    NCK(launch_conv_auto(32, 16, false, o, M->sms, M->err, s));
    return SW_OK;
}

// gradients of the mean squared error of y against target, into dw / db
sw_status backward(sw_model_s *M, int B, int H, int W, const float *target, cudaStream_t s)
{
    Acts &A = M->A;
    const int H1 = H / 2, W1 = W / 2, H2 = H / 4, W2 = W / 4;
    for (int l = 0; l < NLAYERS; ++l) {
        NCK(cudaMemsetAsync(M->dw[l], 0, (size_t)9 * LAYER[l].cout_pad * LAYER[l].cin_pad * 4, s));
        NCK(cudaMemsetAsync(M->db[l], 0, (size_t)LAYER[l].cout_pad * 4, s));
    }
    NCK(cudaMemsetAsync(A.scal + 1, 0, sizeof(double), s));
    NCK(launch_loss(A.y, target, A.gy16, A.scal + 1, B, H, W, s));
    auto wg = [&](int l, const bf16 *g, const bf16 *x, int b_, int h_, int w_) {
        WgradArgs a{g, x, M->dw[l], M->db[l], b_, h_, w_};
        return launch_wgrad_auto(LAYER[l].cin_pad, LAYER[l].cout_pad, a, M->sms, M->err, s);
    };
    // c6 (32 -> 1, padded to 16 outputs)
    NCK(wg(5, A.gy16, A.a5, B, H, W));
    ConvArgs d6 = conv_args(A.gy16, M->wd[5], nullptr, A.gz5, B, H, W, 0);
    d6.mask = A.a5;
    NCK(launch_conv_auto(16, 32, true, d6, M->sms, M->err, s));
    // c5 (96 -> 32) on [up(a4), a1]
    NCK(wg(4, A.gz5, A.cat5, B, H, W));
    NCK(launch_conv_auto(32, 96, true, dgrad_args(A.gz5, M->wd[4], A.gcat5, 96, B, H, W), M->sms, M->err, s));
    NCK(launch_split_up_bwd(A.gcat5, 64, 32, A.a4, A.gz4, A.gskip1, B, H, W, s));
    // c4 (128 -> 64) on [up(a3), a2]
    NCK(wg(3, A.gz4, A.cat4, B, H1, W1));
    NCK(launch_conv_auto(64, 128, true, dgrad_args(A.gz4, M->wd[3], A.gcat4, 128, B, H1, W1), M->sms, M->err, s));
    NCK(launch_split_up_bwd(A.gcat4, 64, 64, A.a3, A.gz3, A.gskip2, B, H1, W1, s));
    // c3 (64 -> 64) on pool(a2)
    NCK(wg(2, A.gz3, A.p2, B, H2, W2));
    NCK(launch_conv_auto(64, 64, true, dgrad_args(A.gz3, M->wd[2], A.gp2, 64, B, H2, W2), M->sms, M->err, s));
    NCK(launch_pool_bwd(A.gskip2, A.gp2, A.a2, A.gz2, B, H1, W1, 64, s));
    // c2 (32 -> 64) on pool(a1)
    NCK(wg(1, A.gz2, A.p1, B, H1, W1));
    NCK(launch_conv_auto(64, 32, true, dgrad_args(A.gz2, M->wd[1], A.gp1, 32, B, H1, W1), M->sms, M->err, s));
    NCK(launch_pool_bwd(A.gskip1, A.gp1, A.a1, A.gz1, B, H, W, 32, s));
    // c1 (4 -> 32, inputs padded to 16)
    NCK(wg(0, A.gz1, A.x0b, B, H, W));
    GradPtrs gp;
    for (int l = 0; l < NLAYERS; ++l) { gp.dw[l] = M->dw[l]; gp.db[l] = M->db[l]; }
    NCK(launch_flatten_grad(gp, M->gflat, s));
    return SW_OK;
}

sw_status pack(sw_model_s *M, cudaStream_t s)
{
    PackArgs a;
    a.master = M->master;
    for (int l = 0; l < NLAYERS; ++l) { a.wf[l] = M->wf[l]; a.wd[l] = M->wd[l]; a.bias[l] = M->bias[l]; }
    NCK(launch_pack(a, s));
    return SW_OK;
}

// ---------------------------------------------------------------------------
// the network's inputs from a grid, and the preconditioner output
// ---------------------------------------------------------------------------
template <class T>
__global__ void k_sumsq(const T *r, size_t n, double *out)
{
    double part = 0.0;
    for (size_t q = blockIdx.x * (size_t)blockDim.x + threadIdx.x; q < n; q += (size_t)gridDim.x * blockDim.x) {
        const double v = (double)r[q];
        part += v * v;
    }
    __shared__ double red[32];
    for (int off = 16; off > 0; off >>= 1) part += __shfl_xor_sync(0xffffffffu, part, off);
    if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = part;
    __syncthreads();
    if (threadIdx.x == 0) {
        double t = 0.0;
        for (int w = 0; w < (int)(blockDim.x >> 5); ++w) t += red[w];
        atomicAdd(out, t);
    }
}

__device__ __forceinline__ float rms_of(const double *sumsq, size_t n)
{
    const double s = sqrt(*sumsq / (double)n);
    return s > 0.0 ? (float)s : 1.f;
}

template <class T>
__global__ void k_features(sw::GridView g, const T *r, const double *sumsq, float *x0)
{
    const int nx = g.nx, ny = g.ny;
    const size_t n = (size_t)nx * ny;
    const float inv = 1.f / rms_of(sumsq, n);
    for (size_t q = blockIdx.x * (size_t)blockDim.x + threadIdx.x; q < n; q += (size_t)gridDim.x * blockDim.x) {
        const int i = (int)(q % nx), j = (int)(q / nx);
        const float d = fabsf(g.wdiag[q]);
        const float axw = g.wax[(size_t)j * nx + (i == 0 ? nx - 1 : i - 1)], axe = g.wax[q];
        const float ayn = g.way[q], ays = j > 0 ? g.way[q - nx] : 0.f;
        const double phi = -M_PI / 2 + (j + 0.5) * M_PI / ny;
        x0[q] = (float)r[q] * inv;
        x0[n + q] = (axw + axe) / d;
        x0[2 * n + q] = (ayn + ays) / d;
        x0[3 * n + q] = (float)sin(phi);
    }
}

__global__ void k_scale_out(sw::GridView g, const float *y, const double *sumsq, float *e)
{
    const size_t n = (size_t)g.nx * g.ny;
    const float s = rms_of(sumsq, n);
    for (size_t q = blockIdx.x * (size_t)blockDim.x + threadIdx.x; q < n; q += (size_t)gridDim.x * blockDim.x)
        e[q] = s * y[q] / fabsf(g.wdiag[q]);
}

__global__ void k_scale_in(sw::GridView g, const float *e, const double *sumsq, float *y)
{
    const size_t n = (size_t)g.nx * g.ny;
    const float inv = 1.f / rms_of(sumsq, n);
    for (size_t q = blockIdx.x * (size_t)blockDim.x + threadIdx.x; q < n; q += (size_t)gridDim.x * blockDim.x)
        y[q] = fabsf(g.wdiag[q]) * e[q] * inv;
}

int grid_blocks(size_t n) { size_t b = (n + 255) / 256; return (int)(b > 2432 ? 2432 : (b < 1 ? 1 : b)); }

template <class T>
sw_status features_t(sw_model_s *M, const sw::GridView &g, const T *r, float *x0, cudaStream_t s)
{
    const size_t n = (size_t)g.nx * g.ny;
    NCK(cudaMemsetAsync(M->A.scal, 0, sizeof(double), s));
    k_sumsq<T><<<grid_blocks(n), 256, 0, s>>>(r, n, M->A.scal);
    k_features<T><<<grid_blocks(n), 256, 0, s>>>(g, r, M->A.scal, x0);
    NCK(cudaGetLastError());
    return SW_OK;
}

} // namespace

// ---------------------------------------------------------------------------
// model entry points used by the solver (sw_api.cu)
// ---------------------------------------------------------------------------
namespace sw {
// e = s y / d for the residual r (FP32 or FP64) of grid g; e FP32 [ny][nx]
sw_status model_precondition(sw_model_s *M, const ::sw_grid_s *grid, const void *r, bool r64, float *e,
                             cudaStream_t s)
{
    const GridView g = grid_view(grid);
    sw_status st = ensure_acts(M, 1, g.ny, g.nx);
    if (st) return st;
    st = r64 ? features_t<double>(M, g, (const double *)r, M->A.x0f, s)
             : features_t<float>(M, g, (const float *)r, M->A.x0f, s);
    if (st) return st;
    if ((st = forward(M, 1, g.ny, g.nx, M->A.x0f, s))) return st;
    k_scale_out<<<grid_blocks((size_t)g.nx * g.ny), 256, 0, s>>>(g, M->A.y, M->A.scal, e);
    NCK(cudaGetLastError());
    return SW_OK;
}

float *model_scratch(sw_model_s *M, int ny, int nx)
{
    if (ensure_acts(M, 1, ny, nx)) return nullptr;
    return M->A.ef;
}

unsigned long long model_gen(sw_model_s *M) { return M->gen; }

sw_status model_check_grid(const ::sw_grid_s *grid)
{
    const GridView g = grid_view(grid);
    return check_shape(1, g.ny, g.nx);
}
} // namespace sw

// ---------------------------------------------------------------------------
// C ABI
// ---------------------------------------------------------------------------
extern "C" sw_status sw_model_create(sw_model *out)
{
    if (!out) return sw::api_fail(SW_ERR_INVALID_ARG, "sw_model_create: out is NULL");
    *out = nullptr;
    if (param_count() != SW_MODEL_PARAMS) return sw::api_fail(SW_ERR_INTERNAL, "parameter count mismatch");
    sw_model_s *M = new (std::nothrow) sw_model_s();
    if (!M) return sw::api_fail(SW_ERR_OOM, "sw_model_create: host allocation failed");
    M->gen = next_model_gen();
    cudaError_t e = cudaGetDevice(&M->device);
    if (e == cudaSuccess) e = cudaDeviceGetAttribute(&M->sms, cudaDevAttrMultiProcessorCount, M->device);
    M->np = param_count();
    size_t bytes = 4 * al256(M->np * 4) + al256(16);
    for (int l = 0; l < NLAYERS; ++l) {
        const size_t nw = (size_t)9 * LAYER[l].cout_pad * LAYER[l].cin_pad;
        bytes += 2 * al256(nw * 2) + al256(nw * 4) + 2 * al256((size_t)LAYER[l].cout_pad * 4);
    }
    if (e == cudaSuccess) e = cudaMalloc(&M->pmem, bytes);
    if (e == cudaSuccess) e = cudaMemset(M->pmem, 0, bytes);
    if (e != cudaSuccess) {
        if (M->pmem) cudaFree(M->pmem);
        delete M;
        return sw::api_fail(e == cudaErrorMemoryAllocation ? SW_ERR_OOM : SW_ERR_CUDA,
                            (std::string("sw_model_create: ") + cudaGetErrorString(e)).c_str());
    }
    char *p = (char *)M->pmem;
    float **f4[] = {&M->master, &M->m, &M->v, &M->gflat};
    for (auto q : f4) { *q = (float *)p; p += al256(M->np * 4); }
    M->err = (int *)p; p += al256(16);
    for (int l = 0; l < NLAYERS; ++l) {
        const size_t nw = (size_t)9 * LAYER[l].cout_pad * LAYER[l].cin_pad;
        M->wf[l] = (bf16 *)p; p += al256(nw * 2);
        M->wd[l] = (bf16 *)p; p += al256(nw * 2);
        M->dw[l] = (float *)p; p += al256(nw * 4);
        M->bias[l] = (float *)p; p += al256((size_t)LAYER[l].cout_pad * 4);
        M->db[l] = (float *)p; p += al256((size_t)LAYER[l].cout_pad * 4);
    }
    *out = M;
    return SW_OK;
}

extern "C" sw_status sw_model_destroy(sw_model M)
{
    if (!M) return sw::api_fail(SW_ERR_INVALID_ARG, "sw_model_destroy: NULL model");
    cudaFree(M->pmem);
    if (M->A.mem) cudaFree(M->A.mem);
    delete M;
    return SW_OK;
}

extern "C" sw_status sw_model_set_params(sw_model M, const float *params)
{
    if (!M || !params) return sw::api_fail(SW_ERR_INVALID_ARG, "sw_model_set_params: NULL argument");
    NCK(cudaMemcpy(M->master, params, M->np * 4, cudaMemcpyHostToDevice));
    NCK(cudaMemset(M->m, 0, M->np * 4));
    NCK(cudaMemset(M->v, 0, M->np * 4));
    M->t = 0;
    sw_status st = pack(M, 0);
    if (st) return st;
    NCK(cudaDeviceSynchronize());
    return SW_OK;
}

extern "C" sw_status sw_model_get_params(sw_model M, float *params)
{
    if (!M || !params) return sw::api_fail(SW_ERR_INVALID_ARG, "sw_model_get_params: NULL argument");
    NCK(cudaDeviceSynchronize());
    NCK(cudaMemcpy(params, M->master, M->np * 4, cudaMemcpyDeviceToHost));
    return SW_OK;
}

extern "C" sw_status sw_model_features(sw_model M, sw_grid g, const float *r, float *x0, void *stream)
{
    if (!M || !g || !r || !x0) return sw::api_fail(SW_ERR_INVALID_ARG, "sw_model_features: NULL argument");
    const sw::GridView v = sw::grid_view(g);
    sw_status st = ensure_acts(M, 1, v.ny, v.nx);
    if (st) return st;
    return features_t<float>(M, v, r, x0, (cudaStream_t)stream);
}

extern "C" sw_status sw_model_forward(sw_model M, int batch, int ny, int nx, const float *x0, float *y, void *stream)
{
    if (!M || !x0 || !y) return sw::api_fail(SW_ERR_INVALID_ARG, "sw_model_forward: NULL argument");
    sw_status st = check_shape(batch, ny, nx);
    if (st) return st;
    if ((st = ensure_acts(M, batch, ny, nx))) return st;
    cudaStream_t s = (cudaStream_t)stream;
    if ((st = forward(M, batch, ny, nx, x0, s))) return st;
    NCK(cudaMemcpyAsync(y, M->A.y, (size_t)batch * ny * nx * 4, cudaMemcpyDeviceToDevice, s));
    return SW_OK;
}

extern "C" sw_status sw_model_loss_grad(sw_model M, int batch, int ny, int nx, const float *x0, const float *target,
                                        double *loss, float *grad, void *stream)
{
    if (!M || !x0 || !target) return sw::api_fail(SW_ERR_INVALID_ARG, "sw_model_loss_grad: NULL argument");
    sw_status st = check_shape(batch, ny, nx);
    if (st) return st;
    if ((st = ensure_acts(M, batch, ny, nx))) return st;
    cudaStream_t s = (cudaStream_t)stream;
    if ((st = forward(M, batch, ny, nx, x0, s))) return st;
    if ((st = backward(M, batch, ny, nx, target, s))) return st;
    if (loss) NCK(cudaMemcpyAsync(loss, M->A.scal + 1, sizeof(double), cudaMemcpyDeviceToHost, s));
    if (grad) NCK(cudaMemcpyAsync(grad, M->gflat, M->np * 4, cudaMemcpyDeviceToHost, s));
    NCK(cudaStreamSynchronize(s));
    return check_err(M);
}

extern "C" sw_status sw_model_train_step(sw_model M, int batch, int ny, int nx, const float *x0, const float *target,
                                         const sw_adamw *hp, double *loss, void *stream)
{
    if (!M || !x0 || !target || !hp) return sw::api_fail(SW_ERR_INVALID_ARG, "sw_model_train_step: NULL argument");
    if (!(hp->lr >= 0) || !(hp->beta1 >= 0 && hp->beta1 < 1) || !(hp->beta2 >= 0 && hp->beta2 < 1) || !(hp->eps > 0))
        return sw::api_fail(SW_ERR_INVALID_ARG, "sw_model_train_step: bad AdamW hyper-parameters");
    sw_status st = check_shape(batch, ny, nx);
    if (st) return st;
    if ((st = ensure_acts(M, batch, ny, nx))) return st;
    cudaStream_t s = (cudaStream_t)stream;
    if ((st = forward(M, batch, ny, nx, x0, s))) return st;
    if ((st = backward(M, batch, ny, nx, target, s))) return st;
    M->t += 1;
    NCK(launch_adamw(M->master, M->m, M->v, M->gflat, M->np, (float)hp->lr, (float)hp->beta1, (float)hp->beta2,
                     (float)hp->eps, (float)hp->weight_decay, M->t, s));
    if ((st = pack(M, s))) return st;
    if (loss) {
        NCK(cudaMemcpyAsync(loss, M->A.scal + 1, sizeof(double), cudaMemcpyDeviceToHost, s));
        NCK(cudaStreamSynchronize(s));
        return check_err(M);
    }
    return SW_OK;
}

extern "C" sw_status sw_model_target(sw_model M, sw_grid g, const float *r, const float *e, float *y, void *stream)
{
    if (!M || !g || !r || !e || !y) return sw::api_fail(SW_ERR_INVALID_ARG, "sw_model_target: NULL argument");
    const sw::GridView v = sw::grid_view(g);
    sw_status st = ensure_acts(M, 1, v.ny, v.nx);
    if (st) return st;
    cudaStream_t s = (cudaStream_t)stream;
    const size_t n = (size_t)v.nx * v.ny;
    NCK(cudaMemsetAsync(M->A.scal, 0, sizeof(double), s));
    k_sumsq<float><<<grid_blocks(n), 256, 0, s>>>(r, n, M->A.scal);
    k_scale_in<<<grid_blocks(n), 256, 0, s>>>(v, e, M->A.scal, y);
    NCK(cudaGetLastError());
    return SW_OK;
}

extern "C" sw_status sw_model_apply(sw_model M, sw_grid g, const float *r, float *e, void *stream)
{
    if (!M || !g || !r || !e) return sw::api_fail(SW_ERR_INVALID_ARG, "sw_model_apply: NULL argument");
    sw_status st = sw::model_check_grid(g);
    if (st) return st;
    return sw::model_precondition(M, g, r, false, e, (cudaStream_t)stream);
}
