// Wake surrogate: a small multilayer perceptron that maps (x/D, y/D, z/D, TSR,
// yaw, U_hub) to the time-mean velocity (u, v, w)/U_hub behind a rotor, used
// to warm-start lattice runs.  Layers: n_in -> n_hidden (x n_layers) -> n_out,
// GELU (x Phi(x), exact erf form) after every hidden layer, linear output.
//
// Weights are kept as FP32 master copies for the optimiser and as BF16 copies
// that the forward and backward products read; every product accumulates in
// FP32.  Kernels: a tiled dense layer (forward and the input-gradient product),
// a per-chunk weight-gradient product with a fixed-order reduction (training
// is deterministic), and Adam.  Parameter layout (FP32, host and device): for
// each layer l, W_l [out][in] row-major, then b_l [out].
#include "lbm_gb300.h"

#include <cuda_bf16.h>
#include <cuda_runtime.h>

#include <cmath>
#include <string>
#include <vector>

namespace mlpgb {

constexpr int kMaxWidth = 128;
constexpr int kTileS = 64;     // samples per CTA in the dense products
constexpr int kChunkS = 64;    // samples per weight-gradient partial
constexpr size_t kDenseSmem = sizeof(float) * (kTileS + kMaxWidth) * (kMaxWidth + 1);
constexpr size_t kWgradSmem = sizeof(float) * kChunkS * (kMaxWidth + 1);

__device__ __forceinline__ float gelu(float z) { return 0.5f * z * (1.0f + erff(z * 0.70710678118654752f)); }

__device__ __forceinline__ float gelu_grad(float z)
{
    const float Phi = 0.5f * (1.0f + erff(z * 0.70710678118654752f));
    const float phi = 0.39894228040143268f * expf(-0.5f * z * z);
    return Phi + z * phi;
}

// Y[s][o] = act(sum_i X[s][i] W[o][i] + b[o]) for a tile of kTileS samples;
// Z (pre-activation) stored when non-null.  256 threads: thread (tx, ty)
// computes outputs o = tx + 32 m (m < 4) for samples s = ty + 8 k (k < 8).
// TRANS: use W^T ([in][out] read as [o][i] with o, i swapped) and multiply by
// act'(Zin) of the incoming gradient (the input-gradient product).
template <bool ACT, bool TRANS>
__global__ void __launch_bounds__(256) k_dense(const float* __restrict__ X, const __nv_bfloat16* __restrict__ W,
                                               const float* __restrict__ bias, float* __restrict__ Z,
                                               float* __restrict__ Y, int B, int I, int O,
                                               const float* __restrict__ Zin)
{
    extern __shared__ float smem[];
    float (*sX)[kMaxWidth + 1] = reinterpret_cast<float (*)[kMaxWidth + 1]>(smem);
    float (*sW)[kMaxWidth + 1] = reinterpret_cast<float (*)[kMaxWidth + 1]>(smem + kTileS * (kMaxWidth + 1));  // [o][i]
    const int tid = threadIdx.y * 32 + threadIdx.x;
    const int s0 = blockIdx.x * kTileS;
    for (int k = tid; k < kTileS * I; k += 256) {
        const int s = k / I, i = k - s * I;
        float v = 0.0f;
        if (s0 + s < B) {
            v = X[(size_t)(s0 + s) * I + i];
            if (TRANS && Zin) v *= gelu_grad(Zin[(size_t)(s0 + s) * I + i]);
        }
        sX[s][i] = v;
    }
    for (int k = tid; k < O * I; k += 256) {
        const int o = k / I, i = k - o * I;
        // forward: W is [O][I]; TRANS: the layer's W is [I][O] (its out = our in)
        sW[o][i] = __bfloat162float(TRANS ? W[(size_t)i * O + o] : W[(size_t)o * I + i]);
    }
    __syncthreads();
    float acc[4][8];
#pragma unroll
    for (int m = 0; m < 4; ++m)
#pragma unroll
        for (int k = 0; k < 8; ++k) acc[m][k] = 0.0f;
    const int tx = threadIdx.x, ty = threadIdx.y;
    for (int i = 0; i < I; ++i) {
        float w[4], xv[8];
#pragma unroll
        for (int m = 0; m < 4; ++m) w[m] = (tx + 32 * m < O) ? sW[tx + 32 * m][i] : 0.0f;
#pragma unroll
        for (int k = 0; k < 8; ++k) xv[k] = sX[ty + 8 * k][i];
#pragma unroll
        for (int m = 0; m < 4; ++m)
#pragma unroll
            for (int k = 0; k < 8; ++k) acc[m][k] = fmaf(xv[k], w[m], acc[m][k]);
    }
#pragma unroll
    for (int m = 0; m < 4; ++m) {
        const int o = tx + 32 * m;
        if (o >= O) continue;
        const float bo = bias ? bias[o] : 0.0f;
#pragma unroll
        for (int k = 0; k < 8; ++k) {
            const int s = s0 + ty + 8 * k;
            if (s >= B) continue;
            const float z = acc[m][k] + bo;
            if (Z) Z[(size_t)s * O + o] = z;
            Y[(size_t)s * O + o] = ACT ? gelu(z) : z;
        }
    }
}

// Weight-gradient partials: for sample chunk c, G_c[o][i] = sum_s dZ[s][o] A[s][i],
// g_c[o] = sum_s dZ[s][o], with dZ = dY * act'(Z) when Z is given.  One CTA per
// chunk, 256 threads striding over the (o, i) pairs.
__global__ void __launch_bounds__(256) k_wgrad_partial(const float* __restrict__ dY, const float* __restrict__ Z,
                                                       const float* __restrict__ A, float* __restrict__ part,
                                                       int B, int I, int O)
{
    extern __shared__ float smem[];
    float (*sD)[kMaxWidth + 1] = reinterpret_cast<float (*)[kMaxWidth + 1]>(smem);
    const int tid = threadIdx.x;
    const int s0 = blockIdx.x * kChunkS;
    const int ns = min(kChunkS, B - s0);
    for (int k = tid; k < ns * O; k += 256) {
        const int s = k / O, o = k - s * O;
        float d = dY[(size_t)(s0 + s) * O + o];
        if (Z) d *= gelu_grad(Z[(size_t)(s0 + s) * O + o]);
        sD[s][o] = d;
    }
    __syncthreads();
    const int nP = O * I + O;
    float* P = part + (size_t)blockIdx.x * nP;
    for (int k = tid; k < nP; k += 256) {
        float acc = 0.0f;
        if (k < O * I) {
            const int o = k / I, i = k - o * I;
            for (int s = 0; s < ns; ++s) acc = fmaf(sD[s][o], A[(size_t)(s0 + s) * I + i], acc);
        } else {
            const int o = k - O * I;
            for (int s = 0; s < ns; ++s) acc += sD[s][o];
        }
        P[k] = acc;
    }
}

// Sum of the chunk partials in chunk order, scaled, into grad.
__global__ void k_wgrad_reduce(const float* __restrict__ part, int n_chunks, int nP, float scale,
                               float* __restrict__ grad)
{
    for (int k = blockIdx.x * blockDim.x + threadIdx.x; k < nP; k += gridDim.x * blockDim.x) {
        float acc = 0.0f;
        for (int c = 0; c < n_chunks; ++c) acc += part[(size_t)c * nP + k];
        grad[k] = acc * scale;
    }
}

// dY = 2 (Y - T) / (B n_out) for the mean squared error; per-sample squared
// errors for the loss.
__global__ void k_mse(const float* __restrict__ Y, const float* __restrict__ T, float* __restrict__ dY,
                      double* __restrict__ sq, int n, float scale)
{
    for (int k = blockIdx.x * blockDim.x + threadIdx.x; k < n; k += gridDim.x * blockDim.x) {
        const float d = Y[k] - T[k];
        dY[k] = scale * d;
        sq[k] = (double)d * (double)d;
    }
}

__global__ void k_sum(const double* __restrict__ v, int n, double* __restrict__ out)
{
    __shared__ double s[256];
    double acc = 0.0;
    for (int k = threadIdx.x; k < n; k += 256) acc += v[k];
    s[threadIdx.x] = acc;
    __syncthreads();
    for (int w = 128; w >= 1; w >>= 1) {
        if (threadIdx.x < w) s[threadIdx.x] += s[threadIdx.x + w];
        __syncthreads();
    }
    if (threadIdx.x == 0) *out = s[0];
}

// Adam (Kingma & Ba 2015) on the FP32 masters; BF16 copies refreshed.
__global__ void k_adam(float* __restrict__ p, const float* __restrict__ g, float* __restrict__ m,
                       float* __restrict__ v, __nv_bfloat16* __restrict__ pb, int n, float lr, float b1, float b2,
                       float eps, float c1, float c2)
{
    for (int k = blockIdx.x * blockDim.x + threadIdx.x; k < n; k += gridDim.x * blockDim.x) {
        const float gk = g[k];
        const float mk = b1 * m[k] + (1.0f - b1) * gk;
        const float vk = b2 * v[k] + (1.0f - b2) * gk * gk;
        m[k] = mk;
        v[k] = vk;
        const float pk = p[k] - lr * (mk / c1) / (sqrtf(vk / c2) + eps);
        p[k] = pk;
        pb[k] = __float2bfloat16_rn(pk);
    }
}

__global__ void k_to_bf16(const float* __restrict__ p, __nv_bfloat16* __restrict__ pb, int n)
{
    for (int k = blockIdx.x * blockDim.x + threadIdx.x; k < n; k += gridDim.x * blockDim.x)
        pb[k] = __float2bfloat16_rn(p[k]);
}

// Gather a minibatch: rows idx[k] of the dataset (idx from splitmix64 of the
// training step and k, modulo the dataset size).
__global__ void k_gather(const float* __restrict__ X, const float* __restrict__ T, int n_data, int I, int O,
                         unsigned long long seed, long long step, int B, float* __restrict__ Xb,
                         float* __restrict__ Tb)
{
    for (int k = blockIdx.x * blockDim.x + threadIdx.x; k < B; k += gridDim.x * blockDim.x) {
        unsigned long long z = seed + ((unsigned long long)step * (unsigned long long)B + (unsigned long long)k + 1ull) *
                                          0x9E3779B97F4A7C15ULL;
        z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ULL;
        z = (z ^ (z >> 27)) * 0x94D049BB133111EBULL;
        z = z ^ (z >> 31);
        const int r = (int)(z % (unsigned long long)n_data);
        for (int i = 0; i < I; ++i) Xb[(size_t)k * I + i] = X[(size_t)r * I + i];
        for (int o = 0; o < O; ++o) Tb[(size_t)k * O + o] = T[(size_t)r * O + o];
    }
}

}  // namespace mlpgb

using namespace mlpgb;

struct mlp_ctx {
    int n_in, width, n_hidden, n_out;
    std::vector<int> fan_in, fan_out;  // per layer
    std::vector<size_t> w_off, b_off;  // offsets into the parameter vector
    int n_param = 0;
    cudaStream_t stream = nullptr;
    float *p = nullptr, *g = nullptr, *m = nullptr, *v = nullptr;
    __nv_bfloat16* pb = nullptr;
    long long adam_t = 0;
    // activations for one batch: A_0 (input) .. A_L, Z_1 .. Z_L
    int cap = 0;
    std::vector<float*> A, Z;
    float *dA = nullptr, *dB = nullptr, *part = nullptr, *T = nullptr, *dY = nullptr;
    double *sq = nullptr, *loss = nullptr;
    float *data_x = nullptr, *data_t = nullptr;
    int n_data = 0;
    std::string err;
    std::vector<void*> allocs;
};

namespace {

lbm_status mlp_fail(mlp_ctx* c, lbm_status s, const std::string& m)
{
    if (c) c->err = m;
    return s;
}

#define MCK(x)                                                                                  \
    do {                                                                                        \
        cudaError_t e_ = (x);                                                                   \
        if (e_ != cudaSuccess) return mlp_fail(c, LBM_ERR_CUDA, std::string(#x) + ": " + cudaGetErrorString(e_)); \
    } while (0)

template <typename T>
T* malloc_dev(mlp_ctx* c, size_t n)
{
    void* p = nullptr;
    if (cudaMalloc(&p, sizeof(T) * (n ? n : 1)) != cudaSuccess) {
        cudaGetLastError();
        return nullptr;
    }
    c->allocs.push_back(p);
    return (T*)p;
}

void free_dev(mlp_ctx* c, void* p)
{
    if (!p) return;
    for (auto it = c->allocs.begin(); it != c->allocs.end(); ++it)
        if (*it == p) {
            c->allocs.erase(it);
            break;
        }
    cudaFree(p);
}

int grid_for(long long n) { return (int)std::min<long long>(std::max<long long>((n + 255) / 256, 1), 152 * 8); }

lbm_status ensure_batch(mlp_ctx* c, int B)
{
    if (B <= c->cap) return LBM_OK;
    const int L = c->n_hidden + 1;
    for (float* a : c->A) free_dev(c, a);
    for (float* z : c->Z) free_dev(c, z);
    free_dev(c, c->dA);
    free_dev(c, c->dB);
    free_dev(c, c->part);
    free_dev(c, c->T);
    free_dev(c, c->dY);
    free_dev(c, c->sq);
    c->cap = 0;  // set again only once every buffer is in place
    c->A.assign(L + 1, nullptr);
    c->Z.assign(L + 1, nullptr);
    c->A[0] = malloc_dev<float>(c, (size_t)B * c->n_in);
    for (int l = 1; l <= L; ++l) {
        c->A[l] = malloc_dev<float>(c, (size_t)B * c->fan_out[l - 1]);
        c->Z[l] = malloc_dev<float>(c, (size_t)B * c->fan_out[l - 1]);
    }
    c->dA = malloc_dev<float>(c, (size_t)B * kMaxWidth);
    c->dB = malloc_dev<float>(c, (size_t)B * kMaxWidth);
    const int n_chunks = (B + kChunkS - 1) / kChunkS;
    c->part = malloc_dev<float>(c, (size_t)n_chunks * (kMaxWidth * kMaxWidth + kMaxWidth));
    c->T = malloc_dev<float>(c, (size_t)B * c->n_out);
    c->dY = malloc_dev<float>(c, (size_t)B * c->n_out);
    c->sq = malloc_dev<double>(c, (size_t)B * c->n_out);
    for (int l = 0; l <= L; ++l)
        if (!c->A[l] || (l > 0 && !c->Z[l])) return mlp_fail(c, LBM_ERR_OOM, "activation allocation failed");
    if (!c->dA || !c->dB || !c->part || !c->T || !c->dY || !c->sq) return mlp_fail(c, LBM_ERR_OOM, "allocation failed");
    c->cap = B;
    return LBM_OK;
}

// Forward pass of B samples already in A[0].
lbm_status forward(mlp_ctx* c, int B)
{
    const int L = c->n_hidden + 1;
    const dim3 grid((B + kTileS - 1) / kTileS), block(32, 8);
    for (int l = 1; l <= L; ++l) {
        const int I = c->fan_in[l - 1], O = c->fan_out[l - 1];
        const __nv_bfloat16* W = c->pb + c->w_off[l - 1];
        const float* b = c->p + c->b_off[l - 1];
        if (l < L)
            k_dense<true, false><<<grid, block, kDenseSmem, c->stream>>>(c->A[l - 1], W, b, c->Z[l], c->A[l], B, I, O,
                                                                        nullptr);
        else
            k_dense<false, false><<<grid, block, kDenseSmem, c->stream>>>(c->A[l - 1], W, b, c->Z[l], c->A[l], B, I, O,
                                                                         nullptr);
        MCK(cudaGetLastError());
    }
    return LBM_OK;
}

// Backward pass from dY (B x n_out) into c->g (gradient of the loss w.r.t. the
// FP32 parameters, products with the BF16 weights).
lbm_status backward(mlp_ctx* c, int B)
{
    const int L = c->n_hidden + 1;
    const int n_chunks = (B + kChunkS - 1) / kChunkS;
    const float* dcur = c->dY;  // gradient w.r.t. A[l] (for l = L: w.r.t. Z[L], linear output)
    float* bufs[2] = {c->dA, c->dB};
    for (int l = L; l >= 1; --l) {
        const int I = c->fan_in[l - 1], O = c->fan_out[l - 1];
        const float* Zl = (l < L) ? c->Z[l] : nullptr;  // hidden layers: dZ = dA * gelu'(Z)
        const int nP = O * I + O;
        k_wgrad_partial<<<n_chunks, 256, kWgradSmem, c->stream>>>(dcur, Zl, c->A[l - 1], c->part, B, I, O);
        MCK(cudaGetLastError());
        k_wgrad_reduce<<<grid_for(nP), 256, 0, c->stream>>>(c->part, n_chunks, nP, 1.0f, c->g + c->w_off[l - 1]);
        MCK(cudaGetLastError());
        if (l > 1) {
            // dA_{l-1} = dZ_l W_l: the dense product with W^T, applying gelu'(Z_l) to the incoming gradient
            float* nxt = bufs[l & 1];
            const dim3 grid((B + kTileS - 1) / kTileS), block(32, 8);
            k_dense<false, true><<<grid, block, kDenseSmem, c->stream>>>(dcur, c->pb + c->w_off[l - 1], nullptr,
                                                                        nullptr, nxt, B, O, I, Zl);
            MCK(cudaGetLastError());
            dcur = nxt;
        }
    }
    return LBM_OK;
}

}  // namespace

extern "C" {

lbm_status mlp_create(int n_in, int width, int n_hidden, int n_out, void* cuda_stream, mlp_ctx** out)
{
    if (!out || n_in < 1 || n_in > kMaxWidth || width < 1 || width > kMaxWidth || n_hidden < 1 || n_hidden > 16 ||
        n_out < 1 || n_out > kMaxWidth)
        return LBM_ERR_INVALID_ARG;
    mlp_ctx* c = new mlp_ctx();
    c->n_in = n_in;
    c->width = width;
    c->n_hidden = n_hidden;
    c->n_out = n_out;
    c->stream = (cudaStream_t)cuda_stream;
    size_t off = 0;
    for (int l = 0; l <= n_hidden; ++l) {
        const int I = l == 0 ? n_in : width, O = l == n_hidden ? n_out : width;
        c->fan_in.push_back(I);
        c->fan_out.push_back(O);
        c->w_off.push_back(off);
        off += (size_t)I * O;
        c->b_off.push_back(off);
        off += O;
    }
    c->n_param = (int)off;
    if (cudaFuncSetAttribute(k_dense<true, false>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kDenseSmem) !=
            cudaSuccess ||
        cudaFuncSetAttribute(k_dense<false, false>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kDenseSmem) !=
            cudaSuccess ||
        cudaFuncSetAttribute(k_dense<false, true>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kDenseSmem) !=
            cudaSuccess ||
        cudaFuncSetAttribute(k_wgrad_partial, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kWgradSmem) !=
            cudaSuccess) {
        cudaGetLastError();
        delete c;
        return LBM_ERR_CUDA;
    }
    c->p = malloc_dev<float>(c, off);
    c->g = malloc_dev<float>(c, off);
    c->m = malloc_dev<float>(c, off);
    c->v = malloc_dev<float>(c, off);
    c->pb = malloc_dev<__nv_bfloat16>(c, off);
    c->loss = malloc_dev<double>(c, 1);
    if (!c->p || !c->g || !c->m || !c->v || !c->pb || !c->loss) {
        mlp_destroy(c);
        return LBM_ERR_OOM;
    }
    cudaMemsetAsync(c->p, 0, sizeof(float) * off, c->stream);
    cudaMemsetAsync(c->m, 0, sizeof(float) * off, c->stream);
    cudaMemsetAsync(c->v, 0, sizeof(float) * off, c->stream);
    cudaMemsetAsync(c->pb, 0, sizeof(__nv_bfloat16) * off, c->stream);
    *out = c;
    return LBM_OK;
}

void mlp_destroy(mlp_ctx* c)
{
    if (!c) return;
    if (c->stream) cudaStreamSynchronize(c->stream);
    else cudaDeviceSynchronize();
    std::vector<void*> all = c->allocs;
    for (void* p : all) cudaFree(p);
    delete c;
}

const char* mlp_last_error(const mlp_ctx* c) { return c ? c->err.c_str() : "null context"; }

int mlp_num_params(const mlp_ctx* c) { return c ? c->n_param : 0; }

lbm_status mlp_set_params(mlp_ctx* c, const float* params)
{
    if (!c || !params) return LBM_ERR_INVALID_ARG;
    MCK(cudaMemcpyAsync(c->p, params, sizeof(float) * c->n_param, cudaMemcpyHostToDevice, c->stream));
    k_to_bf16<<<grid_for(c->n_param), 256, 0, c->stream>>>(c->p, c->pb, c->n_param);
    MCK(cudaGetLastError());
    MCK(cudaMemsetAsync(c->m, 0, sizeof(float) * c->n_param, c->stream));
    MCK(cudaMemsetAsync(c->v, 0, sizeof(float) * c->n_param, c->stream));
    c->adam_t = 0;
    MCK(cudaStreamSynchronize(c->stream));
    return LBM_OK;
}

lbm_status mlp_get_params(mlp_ctx* c, float* params)
{
    if (!c || !params) return LBM_ERR_INVALID_ARG;
    MCK(cudaMemcpyAsync(params, c->p, sizeof(float) * c->n_param, cudaMemcpyDeviceToHost, c->stream));
    MCK(cudaStreamSynchronize(c->stream));
    return LBM_OK;
}

lbm_status mlp_forward(mlp_ctx* c, const float* x, int B, float* y)
{
    if (!c || !x || !y || B < 1) return LBM_ERR_INVALID_ARG;
    const int chunk = 1 << 18;
    for (int s0 = 0; s0 < B; s0 += chunk) {
        const int nb = std::min(chunk, B - s0);
        lbm_status s = ensure_batch(c, nb);
        if (s != LBM_OK) return s;
        MCK(cudaMemcpyAsync(c->A[0], x + (size_t)s0 * c->n_in, sizeof(float) * nb * c->n_in, cudaMemcpyHostToDevice,
                            c->stream));
        s = forward(c, nb);
        if (s != LBM_OK) return s;
        MCK(cudaMemcpyAsync(y + (size_t)s0 * c->n_out, c->A[c->n_hidden + 1], sizeof(float) * nb * c->n_out,
                            cudaMemcpyDeviceToHost, c->stream));
    }
    MCK(cudaStreamSynchronize(c->stream));
    return LBM_OK;
}

lbm_status mlp_loss_grad(mlp_ctx* c, const float* x, const float* target, int B, double* loss, float* grad)
{
    if (!c || !x || !target || B < 1) return LBM_ERR_INVALID_ARG;
    lbm_status s = ensure_batch(c, B);
    if (s != LBM_OK) return s;
    MCK(cudaMemcpyAsync(c->A[0], x, sizeof(float) * B * c->n_in, cudaMemcpyHostToDevice, c->stream));
    MCK(cudaMemcpyAsync(c->T, target, sizeof(float) * B * c->n_out, cudaMemcpyHostToDevice, c->stream));
    s = forward(c, B);
    if (s != LBM_OK) return s;
    const int n = B * c->n_out;
    k_mse<<<grid_for(n), 256, 0, c->stream>>>(c->A[c->n_hidden + 1], c->T, c->dY, c->sq, n, 2.0f / (float)n);
    MCK(cudaGetLastError());
    k_sum<<<1, 256, 0, c->stream>>>(c->sq, n, c->loss);
    MCK(cudaGetLastError());
    s = backward(c, B);
    if (s != LBM_OK) return s;
    double l = 0.0;
    MCK(cudaMemcpyAsync(&l, c->loss, sizeof(double), cudaMemcpyDeviceToHost, c->stream));
    if (grad) MCK(cudaMemcpyAsync(grad, c->g, sizeof(float) * c->n_param, cudaMemcpyDeviceToHost, c->stream));
    MCK(cudaStreamSynchronize(c->stream));
    if (loss) *loss = l / n;
    return LBM_OK;
}

lbm_status mlp_set_data(mlp_ctx* c, const float* x, const float* target, int n)
{
    if (!c || !x || !target || n < 1) return LBM_ERR_INVALID_ARG;
    free_dev(c, c->data_x);
    free_dev(c, c->data_t);
    c->n_data = 0;  // set again only once the data is on the device
    c->data_x = malloc_dev<float>(c, (size_t)n * c->n_in);
    c->data_t = malloc_dev<float>(c, (size_t)n * c->n_out);
    if (!c->data_x || !c->data_t) return mlp_fail(c, LBM_ERR_OOM, "dataset allocation failed");
    MCK(cudaMemcpyAsync(c->data_x, x, sizeof(float) * n * c->n_in, cudaMemcpyHostToDevice, c->stream));
    MCK(cudaMemcpyAsync(c->data_t, target, sizeof(float) * n * c->n_out, cudaMemcpyHostToDevice, c->stream));
    MCK(cudaStreamSynchronize(c->stream));
    c->n_data = n;
    return LBM_OK;
}

lbm_status mlp_train(mlp_ctx* c, int steps, int batch, double lr, unsigned long long seed, double* last_loss)
{
    if (!c || steps < 1 || batch < 1 || c->n_data < 1 || !(lr > 0.0)) return LBM_ERR_INVALID_ARG;
    lbm_status s = ensure_batch(c, batch);
    if (s != LBM_OK) return s;
    const int n = batch * c->n_out;
    for (int it = 0; it < steps; ++it) {
        k_gather<<<grid_for(batch), 256, 0, c->stream>>>(c->data_x, c->data_t, c->n_data, c->n_in, c->n_out, seed,
                                                        c->adam_t, batch, c->A[0], c->T);
        MCK(cudaGetLastError());
        s = forward(c, batch);
        if (s != LBM_OK) return s;
        k_mse<<<grid_for(n), 256, 0, c->stream>>>(c->A[c->n_hidden + 1], c->T, c->dY, c->sq, n, 2.0f / (float)n);
        MCK(cudaGetLastError());
        s = backward(c, batch);
        if (s != LBM_OK) return s;
        c->adam_t++;
        const float b1 = 0.9f, b2 = 0.999f;
        const float c1 = 1.0f - (float)std::pow(0.9, (double)c->adam_t), c2 = 1.0f - (float)std::pow(0.999, (double)c->adam_t);
        k_adam<<<grid_for(c->n_param), 256, 0, c->stream>>>(c->p, c->g, c->m, c->v, c->pb, c->n_param, (float)lr, b1, b2,
                                                            1e-8f, c1, c2);
        MCK(cudaGetLastError());
    }
    if (last_loss) {
        k_sum<<<1, 256, 0, c->stream>>>(c->sq, n, c->loss);
        MCK(cudaGetLastError());
        double l = 0.0;
        MCK(cudaMemcpyAsync(&l, c->loss, sizeof(double), cudaMemcpyDeviceToHost, c->stream));
        MCK(cudaStreamSynchronize(c->stream));
        *last_loss = l / n;
    } else {
        MCK(cudaStreamSynchronize(c->stream));
    }
    return LBM_OK;
}

}  // extern "C"
