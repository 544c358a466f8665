// Learned (p, L) proposer: a small MLP trained on the FMM's own measured
// errors (the error trends of Sec. 5 -- error falls with p at fixed l, and the
// kernel-substitution floor of Sec. 4.1 rises as leaves shrink relative to
// sigma -- learned from runs instead of read off plots).
//
// Network 12 -> 128 -> 128 -> 128 -> 2, SiLU activations; weights in BF16
// (FP32 master copies for the optimiser), biases, activations and all
// accumulation in FP32.  Inputs and outputs are standardised with constants
// held by the model.  Kernels: forward (one CTA per row, one thread per
// output unit), backward (input gradients per (row, unit), weight gradients
// per weight, summed over the batch), MSE loss, Adam.  Features: per-leaf
// counts and circulation sums of the particles at a candidate depth,
// reduced on the device to 12 dimensionless numbers.
#include <cmath>
#include <cstring>
#include <string>
#include <vector>

#include <cuda_bf16.h>

#include "fmm2d_internal.cuh"

namespace {

constexpr int kIn = FMM2D_MLP_INPUTS;    // 12
constexpr int kHid = 128;
constexpr int kOut = FMM2D_MLP_OUTPUTS;  // 2
constexpr int kLayers = 4;
constexpr int kDims[kLayers + 1] = {kIn, kHid, kHid, kHid, kOut};

// parameter offsets in the flat master array: W_l (out x in) then b_l
struct Offsets {
    int w[kLayers], b[kLayers], total;
};
constexpr Offsets offsets() {
    Offsets o{};
    int at = 0;
    for (int l = 0; l < kLayers; ++l) {
        o.w[l] = at;
        at += kDims[l + 1] * kDims[l];
        o.b[l] = at;
        at += kDims[l + 1];
    }
    o.total = at;
    return o;
}
constexpr Offsets kOff = offsets();
static_assert(kOff.total == FMM2D_MLP_PARAMS, "parameter count");

__device__ __forceinline__ float silu(float z) { return z / (1.0f + __expf(-z)); }
__device__ __forceinline__ float silu_grad(float z) {
    float s = 1.0f / (1.0f + __expf(-z));
    return s * (1.0f + z * (1.0f - s));
}

struct Norm {
    float in_mean[kIn], in_std[kIn], out_mean[kOut], out_std[kOut];
};

// out[r][o] = act(sum_i in[r][i] W[o][i] + b[o]); one CTA per row.  For the
// first layer the raw input is standardised; pre-activations are kept for
// the backward pass.
__global__ void linear_fwd_kernel(int rows, int nin, int nout, const float* __restrict__ in,
                                  const __nv_bfloat16* __restrict__ W,
                                  const float* __restrict__ bias, float* __restrict__ z,
                                  float* __restrict__ out, int act, const Norm* __restrict__ norm,
                                  int standardise_in, int unstandardise_out) {
    __shared__ float row[kHid];
    const int r = blockIdx.x;
    if (r >= rows) return;
    for (int i = threadIdx.x; i < nin; i += blockDim.x) {
        float v = in[(int64_t)r * nin + i];
        if (standardise_in) v = (v - norm->in_mean[i]) / norm->in_std[i];
        row[i] = v;
    }
    __syncthreads();
    for (int o = threadIdx.x; o < nout; o += blockDim.x) {
        float acc = bias[o];
        const __nv_bfloat16* w = W + (int64_t)o * nin;
        for (int i = 0; i < nin; ++i) acc = fmaf(row[i], __bfloat162float(w[i]), acc);
        if (z) z[(int64_t)r * nout + o] = acc;
        float v = act ? silu(acc) : acc;
        if (unstandardise_out) v = v * norm->out_std[o] + norm->out_mean[o];
        out[(int64_t)r * nout + o] = v;
    }
}

// dY = 2 (Y - T) / (rows * nout) in standardised units; loss accumulated.
__global__ void mse_kernel(int rows, const float* __restrict__ y, const float* __restrict__ t,
                           const Norm* __restrict__ norm, float* __restrict__ dy,
                           float* __restrict__ loss) {
    int k = blockIdx.x * blockDim.x + threadIdx.x;
    float l = 0.f;
    if (k < rows * kOut) {
        int o = k % kOut;
        float target = (t[k] - norm->out_mean[o]) / norm->out_std[o];
        float d = y[k] - target;
        dy[k] = 2.0f * d / (float)(rows * kOut);
        l = d * d / (float)(rows * kOut);
    }
    for (int s = 16; s > 0; s >>= 1) l += __shfl_xor_sync(0xffffffffu, l, s);
    if ((threadIdx.x & 31) == 0) atomicAdd(loss, l);
}

// dIn[r][i] = sum_o dZ[r][o] W[o][i], times silu'(z_prev) when the previous
// layer is activated.
__global__ void linear_bwd_input_kernel(int rows, int nin, int nout, const float* __restrict__ dz,
                                        const __nv_bfloat16* __restrict__ W,
                                        const float* __restrict__ z_prev,
                                        float* __restrict__ dz_prev) {
    int64_t k = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (k >= (int64_t)rows * nin) return;
    int r = (int)(k / nin), i = (int)(k % nin);
    float acc = 0.f;
    for (int o = 0; o < nout; ++o)
        acc = fmaf(dz[(int64_t)r * nout + o], __bfloat162float(W[(int64_t)o * nin + i]), acc);
    dz_prev[k] = acc * silu_grad(z_prev[k]);
}

// dW[o][i] = sum_r dZ[r][o] in[r][i]; db[o] = sum_r dZ[r][o].
__global__ void linear_bwd_weight_kernel(int rows, int nin, int nout, const float* __restrict__ dz,
                                         const float* __restrict__ in,
                                         float* __restrict__ dW, float* __restrict__ db) {
    int64_t k = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (k < (int64_t)nout * nin) {
        int o = (int)(k / nin), i = (int)(k % nin);
        float acc = 0.f;
        for (int r = 0; r < rows; ++r)
            acc = fmaf(dz[(int64_t)r * nout + o], in[(int64_t)r * nin + i], acc);
        dW[k] = acc;
    } else if (k < (int64_t)nout * nin + nout) {
        int o = (int)(k - (int64_t)nout * nin);
        float acc = 0.f;
        for (int r = 0; r < rows; ++r) acc += dz[(int64_t)r * nout + o];
        db[o] = acc;
    }
}

// Standardised first-layer input (the backward pass of layer 0 needs it).
__global__ void standardise_kernel(int rows, const float* __restrict__ x, const Norm* norm,
                                   float* __restrict__ xs) {
    int k = blockIdx.x * blockDim.x + threadIdx.x;
    if (k < rows * kIn) {
        int i = k % kIn;
        xs[k] = (x[k] - norm->in_mean[i]) / norm->in_std[i];
    }
}

__global__ void adam_kernel(int n, float* __restrict__ w, const float* __restrict__ g,
                            float* __restrict__ m, float* __restrict__ v, float lr, float b1,
                            float b2, float eps, float c1, float c2, __nv_bfloat16* __restrict__ wb,
                            const int* __restrict__ bf16_slot) {
    int k = blockIdx.x * blockDim.x + threadIdx.x;
    if (k >= n) return;
    float gk = g[k];
    float mk = b1 * m[k] + (1.f - b1) * gk;
    float vk = b2 * v[k] + (1.f - b2) * gk * gk;
    m[k] = mk;
    v[k] = vk;
    float wk = w[k] - lr * (mk / c1) / (sqrtf(vk / c2) + eps);
    w[k] = wk;
    int slot = bf16_slot[k];
    if (slot >= 0) wb[slot] = __float2bfloat16_rn(wk);
}

__global__ void to_bf16_kernel(int n, const float* __restrict__ w, __nv_bfloat16* __restrict__ wb,
                               const int* __restrict__ bf16_slot) {
    int k = blockIdx.x * blockDim.x + threadIdx.x;
    if (k < n && bf16_slot[k] >= 0) wb[bf16_slot[k]] = __float2bfloat16_rn(w[k]);
}

// Features: per-leaf counts and circulation sums at depth L, then moments.
__global__ void leaf_hist_kernel(int64_t n, const float* __restrict__ xy,
                                 const float* __restrict__ gamma, double x0, double y0,
                                 double scale, int L, unsigned int* __restrict__ cnt,
                                 double* __restrict__ gsum, double* __restrict__ totals) {
    double sg = 0.0, sa = 0.0;
    const double top = ldexp(1.0, L) - 1.0;
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n;
         i += (int64_t)gridDim.x * blockDim.x) {
        double fx = floor(((double)xy[2 * i] - x0) * scale), fy = floor(((double)xy[2 * i + 1] - y0) * scale);
        fx = fx >= 0.0 ? (fx <= top ? fx : top) : 0.0;  // NaN lands in leaf 0
        fy = fy >= 0.0 ? (fy <= top ? fy : top) : 0.0;
        uint32_t k = fmm2d::morton_key((uint32_t)fx, (uint32_t)fy);
        atomicAdd(&cnt[k], 1u);
        atomicAdd(&gsum[k], (double)gamma[i]);
        sg += gamma[i];
        sa += fabs((double)gamma[i]);
    }
    for (int s = 16; s > 0; s >>= 1) {
        sg += __shfl_xor_sync(0xffffffffu, sg, s);
        sa += __shfl_xor_sync(0xffffffffu, sa, s);
    }
    if ((threadIdx.x & 31) == 0) {
        atomicAdd(&totals[0], sg);
        atomicAdd(&totals[1], sa);
    }
}

// totals[2..8]: sum c, sum c^2, max c, sum S, sum S^2, max |S|, sum |S| over
// leaves (c = particles in the leaf, S = their circulation sum)
__global__ void leaf_moments_kernel(int nleaf, const unsigned int* __restrict__ cnt,
                                    const double* __restrict__ gsum, double* __restrict__ totals) {
    double c1 = 0, c2 = 0, s1 = 0, s2 = 0, cmax = 0, smax = 0, sa = 0;
    for (int k = blockIdx.x * blockDim.x + threadIdx.x; k < nleaf; k += gridDim.x * blockDim.x) {
        double c = cnt[k], s = gsum[k];
        c1 += c;
        c2 += c * c;
        cmax = fmax(cmax, c);
        s1 += s;
        s2 += s * s;
        smax = fmax(smax, fabs(s));
        sa += fabs(s);
    }
    for (int o = 16; o > 0; o >>= 1) {
        c1 += __shfl_xor_sync(0xffffffffu, c1, o);
        c2 += __shfl_xor_sync(0xffffffffu, c2, o);
        s1 += __shfl_xor_sync(0xffffffffu, s1, o);
        s2 += __shfl_xor_sync(0xffffffffu, s2, o);
        sa += __shfl_xor_sync(0xffffffffu, sa, o);
        cmax = fmax(cmax, __shfl_xor_sync(0xffffffffu, cmax, o));
        smax = fmax(smax, __shfl_xor_sync(0xffffffffu, smax, o));
    }
    if ((threadIdx.x & 31) == 0) {
        atomicAdd(&totals[2], c1);
        atomicAdd(&totals[3], c2);
        atomicMax(reinterpret_cast<unsigned long long*>(&totals[4]),
                  (unsigned long long)__double_as_longlong(cmax));
        atomicAdd(&totals[5], s1);
        atomicAdd(&totals[6], s2);
        atomicMax(reinterpret_cast<unsigned long long*>(&totals[7]),
                  (unsigned long long)__double_as_longlong(smax));
        atomicAdd(&totals[8], sa);
    }
}

thread_local std::string g_mlp_error;
fmm2d_status mfail(fmm2d_status s, const std::string& m) {
    g_mlp_error = m;
    return s;
}
#define MCK(call)                                                                        \
    do {                                                                                 \
        cudaError_t e_ = (call);                                                         \
        if (e_ != cudaSuccess)                                                           \
            return mfail(FMM2D_CUDA_ERROR, std::string(#call) + ": " + cudaGetErrorString(e_)); \
    } while (0)

}  // namespace

struct fmm2d_mlp {
    int max_rows = 0;
    int64_t step = 0;
    void* ws = nullptr;
    float* w = nullptr;      // master parameters (FP32)
    float* g = nullptr;      // gradients
    float* m = nullptr;      // Adam moments
    float* v = nullptr;
    __nv_bfloat16* wb = nullptr;  // BF16 weight matrices
    int* slot = nullptr;          // master index -> BF16 slot (-1 for biases)
    Norm* norm = nullptr;
    float* xs = nullptr;          // standardised input
    float* z[kLayers] = {};       // pre-activations
    float* h[kLayers] = {};       // activations (h[3] = output)
    float* dz[kLayers] = {};
    float* loss = nullptr;
    float* feat_ws = nullptr;     // feature scratch
    int bf16_off[kLayers] = {};
};

extern "C" {

const char* fmm2d_mlp_last_error(void) { return g_mlp_error.c_str(); }

fmm2d_status fmm2d_mlp_create(fmm2d_mlp** out, int max_rows, uint64_t seed) {
    if (!out) return mfail(FMM2D_INVALID_ARG, "null output");
    *out = nullptr;
    if (max_rows < 1 || max_rows > (1 << 20)) return mfail(FMM2D_INVALID_ARG, "max_rows");
    auto* n = new fmm2d_mlp();
    n->max_rows = max_rows;
    const int P = kOff.total;
    int nw = 0;
    for (int l = 0; l < kLayers; ++l) {
        n->bf16_off[l] = nw;
        nw += kDims[l + 1] * kDims[l];
    }
    size_t act = 0;
    for (int l = 0; l < kLayers; ++l) act += (size_t)max_rows * kDims[l + 1];
    size_t bytes = (size_t)P * 4 * 4 + (size_t)nw * 2 + (size_t)P * 4 + sizeof(Norm) +
                   (size_t)max_rows * kIn * 4 + act * 4 * 3 + 256 + 64 * 4096;
    if (cudaMalloc(&n->ws, bytes) != cudaSuccess) {
        delete n;
        return mfail(FMM2D_OUT_OF_MEMORY, "mlp workspace");
    }
    char* p = static_cast<char*>(n->ws);
    auto take = [&](size_t b) {
        char* r = p;
        p += (b + 255) & ~(size_t)255;
        return r;
    };
    n->w = (float*)take(P * 4);
    n->g = (float*)take(P * 4);
    n->m = (float*)take(P * 4);
    n->v = (float*)take(P * 4);
    n->wb = (__nv_bfloat16*)take((size_t)nw * 2);
    n->slot = (int*)take(P * 4);
    n->norm = (Norm*)take(sizeof(Norm));
    n->xs = (float*)take((size_t)max_rows * kIn * 4);
    for (int l = 0; l < kLayers; ++l) {
        n->z[l] = (float*)take((size_t)max_rows * kDims[l + 1] * 4);
        n->h[l] = (float*)take((size_t)max_rows * kDims[l + 1] * 4);
        n->dz[l] = (float*)take((size_t)max_rows * kDims[l + 1] * 4);
    }
    n->loss = (float*)take(256);
    n->feat_ws = (float*)take(64 * 4096);
    // initial parameters: uniform(-1/sqrt(fan_in), 1/sqrt(fan_in)) from a
    // splitmix64 stream; biases zero
    std::vector<float> w(P, 0.f);
    std::vector<int> slot(P, -1);
    uint64_t st = seed;
    auto next = [&]() {
        uint64_t z = (st += 0x9E3779B97F4A7C15ull);
        z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
        z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
        return z ^ (z >> 31);
    };
    for (int l = 0; l < kLayers; ++l) {
        float a = 1.0f / sqrtf((float)kDims[l]);
        for (int k = 0; k < kDims[l + 1] * kDims[l]; ++k) {
            double u = (double)(next() >> 11) * (1.0 / 9007199254740992.0);
            w[kOff.w[l] + k] = (float)((2.0 * u - 1.0) * a);
            slot[kOff.w[l] + k] = n->bf16_off[l] + k;
        }
    }
    Norm hn;
    for (int i = 0; i < kIn; ++i) {
        hn.in_mean[i] = 0.f;
        hn.in_std[i] = 1.f;
    }
    for (int o = 0; o < kOut; ++o) {
        hn.out_mean[o] = 0.f;
        hn.out_std[o] = 1.f;
    }
    cudaError_t e = cudaMemcpy(n->w, w.data(), P * 4, cudaMemcpyHostToDevice);
    if (e == cudaSuccess) e = cudaMemcpy(n->slot, slot.data(), P * 4, cudaMemcpyHostToDevice);
    if (e == cudaSuccess) e = cudaMemcpy(n->norm, &hn, sizeof(Norm), cudaMemcpyHostToDevice);
    if (e == cudaSuccess) e = cudaMemset(n->m, 0, P * 4);
    if (e == cudaSuccess) e = cudaMemset(n->v, 0, P * 4);
    if (e == cudaSuccess) {
        to_bf16_kernel<<<(P + 255) / 256, 256>>>(P, n->w, n->wb, n->slot);
        e = cudaDeviceSynchronize();
    }
    if (e != cudaSuccess) {
        cudaFree(n->ws);
        delete n;
        return mfail(FMM2D_CUDA_ERROR, "mlp initialisation");
    }
    *out = n;
    return FMM2D_OK;
}

void fmm2d_mlp_destroy(fmm2d_mlp* n) {
    if (!n) return;
    cudaDeviceSynchronize();
    cudaFree(n->ws);
    delete n;
}

fmm2d_status fmm2d_mlp_set_normalization(fmm2d_mlp* n, const float* in_mean, const float* in_std,
                                         const float* out_mean, const float* out_std) {
    if (!n || !in_mean || !in_std || !out_mean || !out_std)
        return mfail(FMM2D_INVALID_ARG, "null argument");
    Norm hn;
    for (int i = 0; i < kIn; ++i) {
        if (!(in_std[i] > 0.f)) return mfail(FMM2D_INVALID_ARG, "input std must be > 0");
        hn.in_mean[i] = in_mean[i];
        hn.in_std[i] = in_std[i];
    }
    for (int o = 0; o < kOut; ++o) {
        if (!(out_std[o] > 0.f)) return mfail(FMM2D_INVALID_ARG, "output std must be > 0");
        hn.out_mean[o] = out_mean[o];
        hn.out_std[o] = out_std[o];
    }
    MCK(cudaMemcpy(n->norm, &hn, sizeof(Norm), cudaMemcpyHostToDevice));
    return FMM2D_OK;
}

fmm2d_status fmm2d_mlp_params(fmm2d_mlp* n, float* get_host, const float* set_host) {
    if (!n) return mfail(FMM2D_INVALID_ARG, "null model");
    const int P = kOff.total;
    if (get_host) MCK(cudaMemcpy(get_host, n->w, P * 4, cudaMemcpyDeviceToHost));
    if (set_host) {
        MCK(cudaMemcpy(n->w, set_host, P * 4, cudaMemcpyHostToDevice));
        to_bf16_kernel<<<(P + 255) / 256, 256>>>(P, n->w, n->wb, n->slot);
        MCK(cudaGetLastError());
        MCK(cudaDeviceSynchronize());
    }
    return FMM2D_OK;
}

static cudaError_t forward(fmm2d_mlp* n, int rows, const float* x, float* y, bool unstd,
                           cudaStream_t s) {
    const float* in = x;
    for (int l = 0; l < kLayers; ++l) {
        const bool last = l == kLayers - 1;
        float* out = last ? (y ? y : n->h[l]) : n->h[l];
        linear_fwd_kernel<<<rows, 128, 0, s>>>(
            rows, kDims[l], kDims[l + 1], in, n->wb + n->bf16_off[l], n->w + kOff.b[l], n->z[l],
            out, last ? 0 : 1, n->norm, l == 0 ? 1 : 0, (last && unstd) ? 1 : 0);
        in = out;
    }
    return cudaGetLastError();
}

fmm2d_status fmm2d_mlp_forward(fmm2d_mlp* n, int rows, const float* x_dev, float* y_dev,
                               cudaStream_t stream) {
    if (!n || !x_dev || !y_dev) return mfail(FMM2D_INVALID_ARG, "null argument");
    if (rows < 0 || rows > n->max_rows) return mfail(FMM2D_INVALID_ARG, "rows > max_rows");
    if (rows == 0) return FMM2D_OK;
    MCK(forward(n, rows, x_dev, y_dev, true, stream));
    return FMM2D_OK;
}

// Forward + backward; gradients of the mean squared error (standardised
// targets) land in n->g.  Returns the loss in *loss_dev when not NULL.
static fmm2d_status backward(fmm2d_mlp* n, int rows, const float* x, const float* t,
                             float* loss_dev, cudaStream_t s) {
    MCK(forward(n, rows, x, nullptr, false, s));
    MCK(cudaMemsetAsync(n->loss, 0, 4, s));
    const int L = kLayers - 1;
    mse_kernel<<<(rows * kOut + 255) / 256, 256, 0, s>>>(rows, n->h[L], t, n->norm, n->dz[L],
                                                        n->loss);
    standardise_kernel<<<(rows * kIn + 255) / 256, 256, 0, s>>>(rows, x, n->norm, n->xs);
    for (int l = L; l >= 0; --l) {
        const float* in = l == 0 ? n->xs : n->h[l - 1];
        int64_t cnt = (int64_t)kDims[l + 1] * kDims[l] + kDims[l + 1];
        linear_bwd_weight_kernel<<<(unsigned)((cnt + 255) / 256), 256, 0, s>>>(
            rows, kDims[l], kDims[l + 1], n->dz[l], in, n->g + kOff.w[l], n->g + kOff.b[l]);
        if (l > 0) {
            int64_t k = (int64_t)rows * kDims[l];
            linear_bwd_input_kernel<<<(unsigned)((k + 255) / 256), 256, 0, s>>>(
                rows, kDims[l], kDims[l + 1], n->dz[l], n->wb + n->bf16_off[l], n->z[l - 1],
                n->dz[l - 1]);
        }
    }
    MCK(cudaGetLastError());
    if (loss_dev) MCK(cudaMemcpyAsync(loss_dev, n->loss, 4, cudaMemcpyDeviceToDevice, s));
    return FMM2D_OK;
}

fmm2d_status fmm2d_mlp_gradients(fmm2d_mlp* n, int rows, const float* x_dev, const float* t_dev,
                                 float* grad_dev, float* loss_dev, cudaStream_t stream) {
    if (!n || !x_dev || !t_dev || !grad_dev) return mfail(FMM2D_INVALID_ARG, "null argument");
    if (rows < 1 || rows > n->max_rows) return mfail(FMM2D_INVALID_ARG, "rows");
    fmm2d_status st = backward(n, rows, x_dev, t_dev, loss_dev, stream);
    if (st != FMM2D_OK) return st;
    MCK(cudaMemcpyAsync(grad_dev, n->g, kOff.total * 4, cudaMemcpyDeviceToDevice, stream));
    return FMM2D_OK;
}

fmm2d_status fmm2d_mlp_train_step(fmm2d_mlp* n, int rows, const float* x_dev, const float* t_dev,
                                  float lr, float* loss_dev, cudaStream_t stream) {
    if (!n || !x_dev || !t_dev) return mfail(FMM2D_INVALID_ARG, "null argument");
    if (rows < 1 || rows > n->max_rows || !(lr > 0.f))
        return mfail(FMM2D_INVALID_ARG, "rows or learning rate");
    fmm2d_status st = backward(n, rows, x_dev, t_dev, loss_dev, stream);
    if (st != FMM2D_OK) return st;
    n->step += 1;
    const float b1 = 0.9f, b2 = 0.999f;
    const float c1 = 1.f - powf(b1, (float)n->step), c2 = 1.f - powf(b2, (float)n->step);
    const int P = kOff.total;
    adam_kernel<<<(P + 255) / 256, 256, 0, stream>>>(P, n->w, n->g, n->m, n->v, lr, b1, b2, 1e-8f,
                                                      c1, c2, n->wb, n->slot);
    MCK(cudaGetLastError());
    return FMM2D_OK;
}

fmm2d_status fmm2d_features(int64_t n, const float* xy_dev, const float* gamma_dev, double sigma,
                            double x0, double y0, double W, int p, int L, float* feat_host,
                            cudaStream_t stream) {
    if (n < 1 || !xy_dev || !gamma_dev || !feat_host || !(sigma > 0) || !(W > 0) || p < 1 ||
        L < 0 || L > 10)
        return mfail(FMM2D_INVALID_ARG, "bad feature arguments");
    const int nleaf = 1 << (2 * L);
    void* buf = nullptr;
    size_t bytes = (size_t)nleaf * 16 + 256;  // counts | pad | sums | totals
    MCK(cudaMallocAsync(&buf, bytes, stream));
    unsigned int* cnt = (unsigned int*)buf;
    double* gs = (double*)((char*)buf + (size_t)nleaf * 8);  // 8-byte aligned for any nleaf
    double* tot = (double*)((char*)buf + (size_t)nleaf * 16);
    MCK(cudaMemsetAsync(buf, 0, bytes, stream));
    const double scale = ldexp(1.0, L) / W;
    leaf_hist_kernel<<<1024, 256, 0, stream>>>(n, xy_dev, gamma_dev, x0, y0, scale, L, cnt, gs,
                                               tot);
    leaf_moments_kernel<<<256, 256, 0, stream>>>(nleaf, cnt, gs, tot);
    double h[9];
    MCK(cudaMemcpyAsync(h, tot, sizeof(h), cudaMemcpyDeviceToHost, stream));
    MCK(cudaFreeAsync(buf, stream));
    MCK(cudaStreamSynchronize(stream));
    const double sum_g = h[0], sum_abs = h[1] > 0 ? h[1] : 1.0;
    const double cmean = h[2] / nleaf, cvar = fmax(h[3] / nleaf - cmean * cmean, 0.0);
    const double A = sum_abs / nleaf;
    const double smean = h[5] / nleaf, svar = fmax(h[6] / nleaf - smean * smean, 0.0);
    const double hspace = W / sqrt((double)n);
    feat_host[0] = (float)p;
    feat_host[1] = (float)L;
    feat_host[2] = (float)(sigma / hspace);
    feat_host[3] = (float)log2((double)n);
    feat_host[4] = (float)log2(fmax(cmean, 1e-3));
    feat_host[5] = (float)(cmean > 0 ? sqrt(cvar) / cmean : 0.0);
    feat_host[6] = (float)(cmean > 0 ? h[4] / cmean : 0.0);
    feat_host[7] = (float)(h[8] / sum_abs);
    feat_host[8] = (float)(sqrt(svar) / A);
    feat_host[9] = (float)(h[7] / A);
    feat_host[10] = (float)(sum_g / sum_abs);
    feat_host[11] = (float)log10(W / ldexp(1.0, L) / sigma);
    return FMM2D_OK;
}

fmm2d_status fmm2d_propose(fmm2d_mlp* net, int ncand, const float* features_host,
                           const double* cost_host, double tol, double margin, int fallback_p,
                           int fallback_L, int* p_out, int* L_out, int* choice_out,
                           float* predicted_host) {
    if (!net || !p_out || !L_out || ncand < 0 ||
        (ncand > 0 && (!features_host || !cost_host)))
        return mfail(FMM2D_INVALID_ARG, "bad proposal arguments");
    if (!(tol > 0) || !(margin >= 0) || fallback_p < 1 || fallback_p > 32 || fallback_L < 0 ||
        fallback_L > 12)
        return mfail(FMM2D_INVALID_ARG, "tolerance, margin or fallback out of range");
    if (ncand > net->max_rows) return mfail(FMM2D_INVALID_ARG, "more candidates than max_rows");
    *p_out = fallback_p;
    *L_out = fallback_L;
    if (choice_out) *choice_out = -1;
    if (ncand == 0) return FMM2D_OK;
    for (int c = 0; c < ncand; ++c) {
        const float pc = features_host[(size_t)c * kIn], Lc = features_host[(size_t)c * kIn + 1];
        if (!(pc >= 1.f && pc <= 32.f && pc == floorf(pc) && Lc >= 0.f && Lc <= 12.f &&
              Lc == floorf(Lc)))
            return mfail(FMM2D_INVALID_ARG, "candidate " + std::to_string(c) +
                                                ": features 0 and 1 must be integral p and L");
    }
    float *dx = nullptr, *dy = nullptr;
    MCK(cudaMalloc(&dx, (size_t)ncand * kIn * 4));
    if (cudaMalloc(&dy, (size_t)ncand * kOut * 4) != cudaSuccess) {
        cudaFree(dx);
        return mfail(FMM2D_OUT_OF_MEMORY, "proposal buffers");
    }
    cudaError_t e = cudaMemcpy(dx, features_host, (size_t)ncand * kIn * 4, cudaMemcpyHostToDevice);
    if (e == cudaSuccess) e = forward(net, ncand, dx, dy, true, 0);
    std::vector<float> y((size_t)ncand * kOut);
    if (e == cudaSuccess) e = cudaMemcpy(y.data(), dy, y.size() * 4, cudaMemcpyDeviceToHost);
    cudaFree(dx);
    cudaFree(dy);
    if (e != cudaSuccess) return mfail(FMM2D_CUDA_ERROR, cudaGetErrorString(e));
    // a candidate qualifies when its predicted max error sits `margin`
    // decades below the tolerance; the cheapest qualifying one wins
    const double want = log10(tol) - margin;
    int best = -1;
    for (int c = 0; c < ncand; ++c) {
        const float pmax = y[(size_t)c * kOut + 1];
        if (predicted_host) {
            predicted_host[2 * c] = y[(size_t)c * kOut];
            predicted_host[2 * c + 1] = pmax;
        }
        if (std::isfinite(pmax) && pmax <= want && std::isfinite(cost_host[c]) &&
            (best < 0 || cost_host[c] < cost_host[best]))
            best = c;
    }
    if (best >= 0) {
        *p_out = (int)features_host[(size_t)best * kIn];
        *L_out = (int)features_host[(size_t)best * kIn + 1];
        if (choice_out) *choice_out = best;
    }
    return FMM2D_OK;
}

}  // extern "C"
