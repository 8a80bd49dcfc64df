// The reaction surrogate's network (8 -> 64 -> 64 -> 8, ReLU hidden layers)
// and its training on the GPU: forward and backward passes over blocks of
// samples, per-block partial gradients reduced in a fixed order (double
// accumulation), Adam, and the loss accumulated in double.  Not part of the
// paper: the learned replacement of the cell-model update.
#include <cuda_runtime.h>

#include <cmath>
#include <cstring>
#include <vector>

#include "bbx_mlp.cuh"

using namespace bbx;

namespace {

constexpr int kSB = 32;        // samples per training block (static shared memory < 48 KB)
constexpr int kThreads = 256;  // threads per training block

__device__ __forceinline__ unsigned long long splitmix64(unsigned long long z) {
    z += 0x9E3779B97F4A7C15ull;
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
    return z ^ (z >> 31);
}

// Row of sample i of a minibatch: the identity (seed 0) or a counter-based
// hash draw with replacement.
__device__ __forceinline__ long long sample_row(long long i, long long n, unsigned long long seed,
                                                unsigned long long step) {
    if (seed == 0) return i;
    return (long long)(splitmix64(seed ^ (step * 0x100000001B3ull + (unsigned long long)i)) % (unsigned long long)n);
}

// Forward and backward for kSB samples of the minibatch: per-block partial
// gradients (float, [gridDim.x][kMlpParams]) and partial loss (double).
__global__ void __launch_bounds__(kThreads) k_mlp_fwd_bwd(const float* __restrict__ P, const float* __restrict__ X,
                                                           const float* __restrict__ T, long long n, int batch,
                                                           unsigned long long seed, unsigned long long step,
                                                           const float* __restrict__ norm, float* __restrict__ gpart,
                                                           double* __restrict__ lpart) {
    __shared__ float W[kMlpParams];
    __shared__ float xs[kSB][8], h1[kSB][64], h2[kSB][64], dy[kSB][8], d2[kSB][64];
    __shared__ double lsum[kThreads / 32];
    const int tid = threadIdx.x;
    for (int i = tid; i < kMlpParams; i += kThreads) W[i] = P[i];
    const float* W1 = W + kOffW1;
    const float* b1 = W + kOffB1;
    const float* W2 = W + kOffW2;
    const float* b2 = W + kOffB2;
    const float* W3 = W + kOffW3;
    const float* b3 = W + kOffB3;
    const int s0 = blockIdx.x * kSB;
    const int ns = min(kSB, batch - s0);
    // normalised inputs
    for (int e = tid; e < kSB * 8; e += kThreads) {
        const int s = e / 8, k = e % 8;
        float v = 0.0f;
        if (s < ns) {
            const long long r = sample_row(s0 + s, n, seed, step);
            v = (X[r * 8 + k] - norm[kNormMuIn + k]) / norm[kNormSdIn + k];
        }
        xs[s][k] = v;
    }
    __syncthreads();
    for (int e = tid; e < kSB * 64; e += kThreads) {
        const int s = e / 64, j = e % 64;
        float z = b1[j];
#pragma unroll
        for (int k = 0; k < 8; ++k) z = fmaf(W1[j * 8 + k], xs[s][k], z);
        h1[s][j] = fmaxf(z, 0.0f);
    }
    __syncthreads();
    for (int e = tid; e < kSB * 64; e += kThreads) {
        const int s = e / 64, j = e % 64;
        float z = b2[j];
#pragma unroll 16
        for (int k = 0; k < 64; ++k) z = fmaf(W2[j * 64 + k], h1[s][k], z);
        h2[s][j] = fmaxf(z, 0.0f);
    }
    __syncthreads();
    // output, loss and dL/dy = 2 (y - t) / (batch * 8)
    double lacc = 0.0;
    const float scale = 2.0f / (float)(batch * 8);
    for (int e = tid; e < kSB * 8; e += kThreads) {
        const int s = e / 8, o = e % 8;
        float g = 0.0f;
        if (s < ns) {
            float y = b3[o];
#pragma unroll 16
            for (int k = 0; k < 64; ++k) y = fmaf(W3[o * 64 + k], h2[s][k], y);
            const long long r = sample_row(s0 + s, n, seed, step);
            const float t = (T[r * 8 + o] - norm[kNormMuOut + o]) / norm[kNormSdOut + o];
            const float d = y - t;
            lacc += (double)d * (double)d;
            g = scale * d;
        }
        dy[s][o] = g;
    }
    for (int off = 16; off > 0; off >>= 1) lacc += __shfl_xor_sync(0xffffffffu, lacc, off);
    if ((tid & 31) == 0) lsum[tid >> 5] = lacc;
    __syncthreads();
    // dL/dz2 = (dy W3) * relu'(z2)
    for (int e = tid; e < kSB * 64; e += kThreads) {
        const int s = e / 64, k = e % 64;
        float g = 0.0f;
#pragma unroll
        for (int o = 0; o < 8; ++o) g = fmaf(dy[s][o], W3[o * 64 + k], g);
        d2[s][k] = h2[s][k] > 0.0f ? g : 0.0f;
    }
    __syncthreads();
    float* gp = gpart + (size_t)blockIdx.x * kMlpParams;
    // gradients of layer 3 and layer 2 (h2 no longer needed after dW3)
    for (int e = tid; e < 8 * 64; e += kThreads) {
        const int o = e / 64, k = e % 64;
        float g = 0.0f;
        for (int s = 0; s < kSB; ++s) g = fmaf(dy[s][o], h2[s][k], g);
        gp[kOffW3 + e] = g;
    }
    for (int o = tid; o < 8; o += kThreads) {
        float g = 0.0f;
        for (int s = 0; s < kSB; ++s) g += dy[s][o];
        gp[kOffB3 + o] = g;
    }
    for (int e = tid; e < 64 * 64; e += kThreads) {
        const int j = e / 64, k = e % 64;
        float g = 0.0f;
        for (int s = 0; s < kSB; ++s) g = fmaf(d2[s][j], h1[s][k], g);
        gp[kOffW2 + e] = g;
    }
    for (int j = tid; j < 64; j += kThreads) {
        float g = 0.0f;
        for (int s = 0; s < kSB; ++s) g += d2[s][j];
        gp[kOffB2 + j] = g;
    }
    __syncthreads();
    // dL/dz1 = (d2 W2) * relu'(z1), written over h2
    for (int e = tid; e < kSB * 64; e += kThreads) {
        const int s = e / 64, k = e % 64;
        float g = 0.0f;
#pragma unroll 16
        for (int j = 0; j < 64; ++j) g = fmaf(d2[s][j], W2[j * 64 + k], g);
        h2[s][k] = h1[s][k] > 0.0f ? g : 0.0f;
    }
    __syncthreads();
    for (int e = tid; e < 64 * 8; e += kThreads) {
        const int j = e / 8, k = e % 8;
        float g = 0.0f;
        for (int s = 0; s < kSB; ++s) g = fmaf(h2[s][j], xs[s][k], g);
        gp[kOffW1 + e] = g;
    }
    for (int j = tid; j < 64; j += kThreads) {
        float g = 0.0f;
        for (int s = 0; s < kSB; ++s) g += h2[s][j];
        gp[kOffB1 + j] = g;
    }
    if (tid == 0) {
        double l = 0.0;
        for (int w = 0; w < kThreads / 32; ++w) l += lsum[w];
        lpart[blockIdx.x] = l;
    }
}

// Sum the per-block gradients in block order (double accumulation), write
// the gradient, and (if lr > 0) apply one Adam step.  Block 0 also sums the
// loss partials: loss = sum / (batch * 8).
__global__ void k_mlp_reduce_adam(const float* __restrict__ gpart, int nblk, const double* __restrict__ lpart,
                                  int batch, float* __restrict__ P, float* __restrict__ M, float* __restrict__ V,
                                  float* __restrict__ G, double* __restrict__ loss, int step, float lr, float beta1,
                                  float beta2, float eps) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i < kMlpParams) {
        double g = 0.0;
        for (int b = 0; b < nblk; ++b) g += gpart[(size_t)b * kMlpParams + i];
        G[i] = (float)g;
        if (lr > 0.0f) {
            const float gf = (float)g;
            const float m = beta1 * M[i] + (1.0f - beta1) * gf;
            const float v = beta2 * V[i] + (1.0f - beta2) * gf * gf;
            M[i] = m;
            V[i] = v;
            const float mh = m / (1.0f - powf(beta1, (float)step));
            const float vh = v / (1.0f - powf(beta2, (float)step));
            P[i] = P[i] - lr * mh / (sqrtf(vh) + eps);
        }
    }
    if (blockIdx.x == 0 && threadIdx.x == 0) {
        double l = 0.0;
        for (int b = 0; b < nblk; ++b) l += lpart[b];
        *loss = l / ((double)batch * 8.0);
    }
}

// Per-feature mean, standard deviation (of inputs and targets) and input
// min/max, accumulated in double by one block.
__global__ void k_mlp_stats(const float* __restrict__ X, const float* __restrict__ T, long long n,
                            double* __restrict__ out /* 8 x {sum_x, sumsq_x, min_x, max_x, sum_t, sumsq_t} */) {
    __shared__ double red[6][8][32];
    const int f = threadIdx.x % 8, lane = threadIdx.x / 8;  // 256 threads: 8 features x 32 lanes
    double sx = 0, sxx = 0, st = 0, stt = 0, mn = 1e300, mx = -1e300;
    for (long long r = lane; r < n; r += 32) {
        const double x = X[r * 8 + f], t = T[r * 8 + f];
        sx += x;
        sxx += x * x;
        st += t;
        stt += t * t;
        mn = fmin(mn, x);
        mx = fmax(mx, x);
    }
    red[0][f][lane] = sx;
    red[1][f][lane] = sxx;
    red[2][f][lane] = mn;
    red[3][f][lane] = mx;
    red[4][f][lane] = st;
    red[5][f][lane] = stt;
    __syncthreads();
    if (threadIdx.x < 8) {
        const int ff = threadIdx.x;
        double a[6] = {0, 0, 1e300, -1e300, 0, 0};
        for (int l = 0; l < 32; ++l) {
            a[0] += red[0][ff][l];
            a[1] += red[1][ff][l];
            a[2] = fmin(a[2], red[2][ff][l]);
            a[3] = fmax(a[3], red[3][ff][l]);
            a[4] += red[4][ff][l];
            a[5] += red[5][ff][l];
        }
        for (int q = 0; q < 6; ++q) out[ff * 6 + q] = a[q];
    }
}

__global__ void k_mlp_init(float* P, unsigned long long seed) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= kMlpParams) return;
    // uniform(-1/sqrt(fan_in), 1/sqrt(fan_in)) weights, zero biases
    float r = 0.0f;
    if (i < kOffB1) r = rsqrtf(8.0f);
    else if (i >= kOffW2 && i < kOffB2) r = 0.125f;
    else if (i >= kOffW3 && i < kOffB3) r = 0.125f;
    const unsigned long long h = splitmix64(seed ^ (unsigned long long)(i + 1) * 0xD1B54A32D192ED03ull);
    const float u = (float)((h >> 40) * (1.0 / 16777216.0));  // [0, 1)
    P[i] = r * (2.0f * u - 1.0f);
}

}  // namespace

struct bbx_mlp {
    cudaStream_t stream = nullptr;
    float* d_P = nullptr;     // parameters, packed W1 b1 W2 b2 W3 b3
    float* d_M = nullptr;     // Adam first moment
    float* d_V = nullptr;     // Adam second moment
    float* d_G = nullptr;     // last gradient
    float* d_gpart = nullptr;
    double* d_lpart = nullptr;
    double* d_loss = nullptr;
    float* d_norm = nullptr;  // kNormSize floats
    float h_norm[kNormSize];
    int cap_blocks = 0;
    int step = 0;
};

namespace {

int ensure_blocks(bbx_mlp* m, int nblk) {
    if (nblk <= m->cap_blocks) return BBX_OK;
    cudaFree(m->d_gpart);
    cudaFree(m->d_lpart);
    m->d_gpart = nullptr;
    m->d_lpart = nullptr;
    if (cudaMalloc(&m->d_gpart, sizeof(float) * kMlpParams * (size_t)nblk) != cudaSuccess ||
        cudaMalloc(&m->d_lpart, sizeof(double) * (size_t)nblk) != cudaSuccess) {
        cudaGetLastError();
        m->cap_blocks = 0;
        return BBX_ERR_NOMEM;
    }
    m->cap_blocks = nblk;
    return BBX_OK;
}

int run_batch(bbx_mlp* m, const float* X, const float* T, long long n, int batch, unsigned long long seed, float lr) {
    const int nblk = (batch + kSB - 1) / kSB;
    int rc = ensure_blocks(m, nblk);
    if (rc) return rc;
    if (lr > 0.0f) ++m->step;
    k_mlp_fwd_bwd<<<nblk, kThreads, 0, m->stream>>>(m->d_P, X, T, n, batch, seed, (unsigned long long)m->step,
                                                    m->d_norm, m->d_gpart, m->d_lpart);
    k_mlp_reduce_adam<<<(kMlpParams + 255) / 256, 256, 0, m->stream>>>(m->d_gpart, nblk, m->d_lpart, batch, m->d_P,
                                                                       m->d_M, m->d_V, m->d_G, m->d_loss, m->step,
                                                                       lr, 0.9f, 0.999f, 1e-8f);
    if (cudaGetLastError() != cudaSuccess) return BBX_ERR_CUDA;
    return BBX_OK;
}

}  // namespace

const float* bbx_mlp_device_params(const bbx_mlp* m) { return m->d_P; }
const float* bbx_mlp_device_norm(const bbx_mlp* m) { return m->d_norm; }

extern "C" {

int bbx_mlp_create(bbx_mlp** out, unsigned long long seed, void* cuda_stream) {
    if (!out) return BBX_ERR_ARG;
    *out = nullptr;
    bbx_mlp* m = new (std::nothrow) bbx_mlp();
    if (!m) return BBX_ERR_NOMEM;
    m->stream = static_cast<cudaStream_t>(cuda_stream);
    if (cudaMalloc(&m->d_P, sizeof(float) * kMlpParams) != cudaSuccess ||
        cudaMalloc(&m->d_M, sizeof(float) * kMlpParams) != cudaSuccess ||
        cudaMalloc(&m->d_V, sizeof(float) * kMlpParams) != cudaSuccess ||
        cudaMalloc(&m->d_G, sizeof(float) * kMlpParams) != cudaSuccess ||
        cudaMalloc(&m->d_loss, sizeof(double)) != cudaSuccess ||
        cudaMalloc(&m->d_norm, sizeof(float) * kNormSize) != cudaSuccess) {
        cudaGetLastError();
        bbx_mlp_destroy(m);
        return BBX_ERR_NOMEM;
    }
    for (int k = 0; k < 8; ++k) {
        m->h_norm[kNormMuIn + k] = 0.0f;
        m->h_norm[kNormSdIn + k] = 1.0f;
        m->h_norm[kNormMuOut + k] = 0.0f;
        m->h_norm[kNormSdOut + k] = 1.0f;
        m->h_norm[kNormLo + k] = -INFINITY;
        m->h_norm[kNormHi + k] = INFINITY;
    }
    k_mlp_init<<<(kMlpParams + 255) / 256, 256, 0, m->stream>>>(m->d_P, seed);
    if (cudaGetLastError() != cudaSuccess ||
        cudaMemsetAsync(m->d_M, 0, sizeof(float) * kMlpParams, m->stream) != cudaSuccess ||
        cudaMemsetAsync(m->d_V, 0, sizeof(float) * kMlpParams, m->stream) != cudaSuccess ||
        cudaMemcpyAsync(m->d_norm, m->h_norm, sizeof(m->h_norm), cudaMemcpyHostToDevice, m->stream) != cudaSuccess ||
        cudaStreamSynchronize(m->stream) != cudaSuccess) {
        cudaGetLastError();
        bbx_mlp_destroy(m);
        return BBX_ERR_CUDA;
    }
    *out = m;
    return BBX_OK;
}

void bbx_mlp_destroy(bbx_mlp* m) {
    if (!m) return;
    cudaStreamSynchronize(m->stream);
    cudaFree(m->d_P);
    cudaFree(m->d_M);
    cudaFree(m->d_V);
    cudaFree(m->d_G);
    cudaFree(m->d_gpart);
    cudaFree(m->d_lpart);
    cudaFree(m->d_loss);
    cudaFree(m->d_norm);
    cudaGetLastError();
    delete m;
}

int bbx_mlp_set_params(bbx_mlp* m, const float* params, size_t n) {
    if (!m || !params || n != (size_t)kMlpParams) return BBX_ERR_ARG;
    if (cudaMemcpyAsync(m->d_P, params, sizeof(float) * kMlpParams, cudaMemcpyHostToDevice, m->stream) != cudaSuccess ||
        cudaMemsetAsync(m->d_M, 0, sizeof(float) * kMlpParams, m->stream) != cudaSuccess ||
        cudaMemsetAsync(m->d_V, 0, sizeof(float) * kMlpParams, m->stream) != cudaSuccess ||
        cudaStreamSynchronize(m->stream) != cudaSuccess) {
        cudaGetLastError();
        return BBX_ERR_CUDA;
    }
    m->step = 0;
    return BBX_OK;
}

int bbx_mlp_get_params(bbx_mlp* m, float* params, size_t n) {
    if (!m || !params || n != (size_t)kMlpParams) return BBX_ERR_ARG;
    if (cudaMemcpyAsync(params, m->d_P, sizeof(float) * kMlpParams, cudaMemcpyDeviceToHost, m->stream) != cudaSuccess ||
        cudaStreamSynchronize(m->stream) != cudaSuccess) {
        cudaGetLastError();
        return BBX_ERR_CUDA;
    }
    return BBX_OK;
}

int bbx_mlp_set_normalization(bbx_mlp* m, const float* norm, size_t n) {
    if (!m || !norm || n != (size_t)kNormSize) return BBX_ERR_ARG;
    for (int k = 0; k < 8; ++k)
        if (!(norm[kNormSdIn + k] > 0.0f) || !(norm[kNormSdOut + k] > 0.0f)) return BBX_ERR_ARG;
    memcpy(m->h_norm, norm, sizeof(m->h_norm));
    if (cudaMemcpyAsync(m->d_norm, m->h_norm, sizeof(m->h_norm), cudaMemcpyHostToDevice, m->stream) != cudaSuccess ||
        cudaStreamSynchronize(m->stream) != cudaSuccess) {
        cudaGetLastError();
        return BBX_ERR_CUDA;
    }
    return BBX_OK;
}

int bbx_mlp_get_normalization(bbx_mlp* m, float* norm, size_t n) {
    if (!m || !norm || n != (size_t)kNormSize) return BBX_ERR_ARG;
    memcpy(norm, m->h_norm, sizeof(m->h_norm));
    return BBX_OK;
}

int bbx_mlp_fit_normalization(bbx_mlp* m, const float* x_dev, const float* t_dev, long long n) {
    if (!m || !x_dev || !t_dev || n < 2) return BBX_ERR_ARG;
    double* d_out = nullptr;
    if (cudaMalloc(&d_out, sizeof(double) * 48) != cudaSuccess) {
        cudaGetLastError();
        return BBX_ERR_NOMEM;
    }
    double h[48];
    k_mlp_stats<<<1, 256, 0, m->stream>>>(x_dev, t_dev, n, d_out);
    cudaError_t e = cudaGetLastError();
    if (e == cudaSuccess) e = cudaMemcpyAsync(h, d_out, sizeof(h), cudaMemcpyDeviceToHost, m->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(m->stream);
    cudaFree(d_out);
    if (e != cudaSuccess) {
        cudaGetLastError();
        return BBX_ERR_CUDA;
    }
    float norm[kNormSize];
    for (int k = 0; k < 8; ++k) {
        const double* a = h + 6 * k;
        const double mx = a[0] / n, vx = a[1] / n - mx * mx;
        const double mt = a[4] / n, vt = a[5] / n - mt * mt;
        norm[kNormMuIn + k] = (float)mx;
        norm[kNormSdIn + k] = (float)std::sqrt(vx > 1e-30 ? vx : 1e-30);
        norm[kNormMuOut + k] = (float)mt;
        norm[kNormSdOut + k] = (float)std::sqrt(vt > 1e-30 ? vt : 1e-30);
        norm[kNormLo + k] = (float)a[2];
        norm[kNormHi + k] = (float)a[3];
    }
    return bbx_mlp_set_normalization(m, norm, kNormSize);
}

int bbx_mlp_gradients(bbx_mlp* m, const float* x_dev, const float* t_dev, int batch, float* grad, size_t n,
                      double* loss) {
    if (!m || !x_dev || !t_dev || batch <= 0 || !grad || n != (size_t)kMlpParams) return BBX_ERR_ARG;
    int rc = run_batch(m, x_dev, t_dev, batch, batch, 0ull, 0.0f);
    if (rc) return rc;
    if (cudaMemcpyAsync(grad, m->d_G, sizeof(float) * kMlpParams, cudaMemcpyDeviceToHost, m->stream) != cudaSuccess ||
        (loss && cudaMemcpyAsync(loss, m->d_loss, sizeof(double), cudaMemcpyDeviceToHost, m->stream) != cudaSuccess) ||
        cudaStreamSynchronize(m->stream) != cudaSuccess) {
        cudaGetLastError();
        return BBX_ERR_CUDA;
    }
    return BBX_OK;
}

int bbx_mlp_train(bbx_mlp* m, const float* x_dev, const float* t_dev, long long n, int batch, int steps, double lr,
                  unsigned long long seed, double* final_loss) {
    if (!m || !x_dev || !t_dev || n <= 0 || batch <= 0 || steps < 0 || !(lr > 0.0) || seed == 0) return BBX_ERR_ARG;
    for (int s = 0; s < steps; ++s) {
        int rc = run_batch(m, x_dev, t_dev, n, batch, seed, (float)lr);
        if (rc) return rc;
    }
    if (final_loss) {
        if (cudaMemcpyAsync(final_loss, m->d_loss, sizeof(double), cudaMemcpyDeviceToHost, m->stream) != cudaSuccess ||
            cudaStreamSynchronize(m->stream) != cudaSuccess) {
            cudaGetLastError();
            return BBX_ERR_CUDA;
        }
    }
    return BBX_OK;
}

}  // extern "C"
