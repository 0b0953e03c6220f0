// The learned stand-in for the Ewald real-space force factor: FP64 targets,
// FP32 training (forward, backward, Adam) and evaluation kernels, packing for
// the tensor-core tile evaluator, and their C entry points.
//
// Training follows the usual reverse-mode rules for
//   L = (1/n) sum_i w_i (y(r_i) - t_i)^2,
//   y = W3 . SiLU(W2 SiLU(W1 x + b1) + b2) + b3,   x = (r - c0) c1,
// with d SiLU(z)/dz = s(z) (1 + z (1 - s(z))), s the logistic function.
// The factor itself, c(r) = erfc(beta r) + 2 beta r / sqrt(pi)
// exp(-beta^2 r^2), is Sec. 3.2's Ewald correction written as the force
// factor of a non-excluded pair (F = f qq c(r) / r^2).
#include <cmath>

#include "nb_internal.cuh"
#include "nb_mlp.cuh"

namespace nbc {

__global__ void k_ewald_factor(const double* __restrict__ r, long long n, double beta, double* __restrict__ out) {
    const double two_over_sqrtpi = 1.1283791670955126;
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x) {
        const double br = beta * r[i];
        out[i] = erfc(br) + two_over_sqrtpi * br * exp(-br * br);
    }
}

// One warp fills the per-lane layout of the tensor-core evaluator.
__global__ void k_mlp_pack(const float* __restrict__ p, float c0, float c1, MlpTC* __restrict__ out) {
    const int lane = threadIdx.x;
    if (lane >= 32) return;
    const int g = lane >> 2, q = lane & 3;
    for (int u = 0; u < 4; ++u) {
        for (int s = 0; s < 2; ++s) {
            const int n = u * 8 + g;
            uint32_t h[2], l[2];
            for (int reg = 0; reg < 2; ++reg) {
                const int k = s * 16 + reg * 8 + 2 * q;
                const float a = p[kMlpW2 + n * kMlpH + k], b = p[kMlpW2 + n * kMlpH + k + 1];
                mlp_split(a, b, h[reg], l[reg]);
            }
            out->bfrag[u * 2 + s][lane] = make_uint4(h[0], h[1], l[0], l[1]);
        }
    }
    float v[4][8];
    for (int m = 0; m < 8; ++m) {
        const int hid = mlp_hidden(m, q);
        v[0][m] = p[kMlpW1 + hid];
        v[1][m] = p[kMlpB1 + hid];
        v[2][m] = p[kMlpB2 + hid];
        v[3][m] = p[kMlpW3 + hid];
    }
    for (int c = 0; c < 4; ++c) {
        out->lanec[2 * c][lane] = make_float4(v[c][0], v[c][1], v[c][2], v[c][3]);
        out->lanec[2 * c + 1][lane] = make_float4(v[c][4], v[c][5], v[c][6], v[c][7]);
    }
    if (lane == 0) {
        out->b3 = p[kMlpB3];
        out->c0 = c0;
        out->c1 = c1;
        out->pad = 0.0f;
    }
}

__device__ __forceinline__ float silu_acc(float z) { return z / (1.0f + expf(-z)); }

__device__ __forceinline__ float silu_grad(float z) {
    const float s = 1.0f / (1.0f + expf(-z));
    return s * (1.0f + z * (1.0f - s));
}

// FP32 forward on the CUDA cores, one thread per sample.
__global__ void __launch_bounds__(256) k_mlp_forward(const float* __restrict__ p, float c0, float c1,
                                                     const float* __restrict__ r, long long n,
                                                     float* __restrict__ y) {
    __shared__ float sP[kMlpParams];
    for (int k = threadIdx.x; k < kMlpParams; k += blockDim.x) sP[k] = p[k];
    __syncthreads();
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x) {
        const float x = (r[i] - c0) * c1;
        float h1[kMlpH];
#pragma unroll
        for (int j = 0; j < kMlpH; ++j) h1[j] = silu_acc(fmaf(sP[kMlpW1 + j], x, sP[kMlpB1 + j]));
        float out = sP[kMlpB3];
        for (int k = 0; k < kMlpH; ++k) {
            float z = sP[kMlpB2 + k];
#pragma unroll
            for (int j = 0; j < kMlpH; ++j) z = fmaf(sP[kMlpW2 + k * kMlpH + j], h1[j], z);
            out = fmaf(sP[kMlpW3 + k], silu_acc(z), out);
        }
        y[i] = out;
    }
}

// Tensor-core forward, one warp per tile of 64 samples (the evaluator the
// force kernel uses).
__global__ void __launch_bounds__(128) k_mlp_forward_tc(const MlpTC* __restrict__ P, const float* __restrict__ r,
                                                        long long n, float* __restrict__ y) {
    __shared__ MlpTC sM;
    {
        const uint4* src = reinterpret_cast<const uint4*>(P);
        uint4* dst = reinterpret_cast<uint4*>(&sM);
        for (int k = threadIdx.x; k < (int)(sizeof(MlpTC) / 16); k += blockDim.x) dst[k] = src[k];
    }
    __syncthreads();
    const int lane = threadIdx.x & 31, g = lane >> 2;
    const long long ntile = (n + 63) / 64;
    for (long long tile = blockIdx.x * (long long)(blockDim.x / 32) + (threadIdx.x >> 5); tile < ntile;
         tile += (long long)gridDim.x * (blockDim.x / 32)) {
#pragma unroll 1
        for (int t = 0; t < 4; ++t) {
            const long long i0 = tile * 64 + 16 * t + g, i1 = i0 + 8;
            const float x0 = ((i0 < n ? r[i0] : sM.c0) - sM.c0) * sM.c1;
            const float x1 = ((i1 < n ? r[i1] : sM.c0) - sM.c0) * sM.c1;
            float o0, o1;
            mlp_mtile(sM, lane, x0, x1, o0, o1);
            if ((lane & 3) == 0) {
                if (i0 < n) y[i0] = o0;
                if (i1 < n) y[i1] = o1;
            }
        }
    }
}

constexpr int kGradThreads = 128;
constexpr int kSmallGrads = 4 * kMlpH + 1;   // W1, b1, b2, W3, b3

// Loss and gradient over samples (start + i) mod n_data, i < batch, scaled by
// inv_n; gradients and loss are added to grad and *loss.
__global__ void __launch_bounds__(kGradThreads) k_mlp_grad(const float* __restrict__ p, float c0, float c1,
                                                           const float* __restrict__ r, const float* __restrict__ t,
                                                           const float* __restrict__ w, long long n_data,
                                                           long long start, long long batch, float inv_n,
                                                           float* __restrict__ grad, float* __restrict__ loss) {
    __shared__ float sP[kMlpParams];
    __shared__ float sH1[kGradThreads][kMlpH + 1];
    __shared__ float sD2[kGradThreads][kMlpH + 1];
    __shared__ float sG[kSmallGrads];
    __shared__ float sLoss;
    for (int k = threadIdx.x; k < kMlpParams; k += blockDim.x) sP[k] = p[k];
    for (int k = threadIdx.x; k < kSmallGrads; k += blockDim.x) sG[k] = 0.0f;
    if (threadIdx.x == 0) sLoss = 0.0f;
    __syncthreads();
    const unsigned full = 0xffffffffu;
    float gw2[kMlpH * kMlpH / kGradThreads];
#pragma unroll
    for (int c = 0; c < kMlpH * kMlpH / kGradThreads; ++c) gw2[c] = 0.0f;
    float lsum = 0.0f;
    for (long long base = (long long)blockIdx.x * kGradThreads; base < batch; base += (long long)gridDim.x * kGradThreads) {
        const long long i = base + threadIdx.x;
        const bool valid = i < batch;
        float x = 0.0f, ti = 0.0f, wi = 0.0f;
        if (valid) {
            const long long s = (start + i) % n_data;
            x = (r[s] - c0) * c1;
            ti = t[s];
            wi = w ? w[s] : 1.0f;
        }
        float h1[kMlpH], z2[kMlpH];
#pragma unroll
        for (int j = 0; j < kMlpH; ++j) h1[j] = silu_acc(fmaf(sP[kMlpW1 + j], x, sP[kMlpB1 + j]));
        float out = sP[kMlpB3];
#pragma unroll
        for (int k = 0; k < kMlpH; ++k) {
            float z = sP[kMlpB2 + k];
#pragma unroll
            for (int j = 0; j < kMlpH; ++j) z = fmaf(sP[kMlpW2 + k * kMlpH + j], h1[j], z);
            z2[k] = z;
            out = fmaf(sP[kMlpW3 + k], silu_acc(z), out);
        }
        const float e = out - ti;
        lsum += valid ? wi * e * e * inv_n : 0.0f;
        const float dy = valid ? 2.0f * wi * e * inv_n : 0.0f;
        // output layer and layer-2 deltas
        float gb3 = dy;
#pragma unroll
        for (int k = 0; k < kMlpH; ++k) {
            const float h2 = silu_acc(z2[k]);
            const float d2 = dy * sP[kMlpW3 + k] * silu_grad(z2[k]);
            z2[k] = d2;   // z2 now holds dL/dz2
            float a = dy * h2, b = d2;
            for (int o = 16; o > 0; o >>= 1) {
                a += __shfl_xor_sync(full, a, o);
                b += __shfl_xor_sync(full, b, o);
            }
            if ((threadIdx.x & 31) == 0) {
                atomicAdd(&sG[3 * kMlpH + k], a);   // W3
                atomicAdd(&sG[2 * kMlpH + k], b);   // b2
            }
        }
        for (int o = 16; o > 0; o >>= 1) gb3 += __shfl_xor_sync(full, gb3, o);
        if ((threadIdx.x & 31) == 0) atomicAdd(&sG[4 * kMlpH], gb3);
        // layer-1 deltas
        for (int j = 0; j < kMlpH; ++j) {
            float dh = 0.0f;
#pragma unroll
            for (int k = 0; k < kMlpH; ++k) dh = fmaf(sP[kMlpW2 + k * kMlpH + j], z2[k], dh);
            const float d1 = dh * silu_grad(fmaf(sP[kMlpW1 + j], x, sP[kMlpB1 + j]));
            float a = d1 * x, b = d1;
            for (int o = 16; o > 0; o >>= 1) {
                a += __shfl_xor_sync(full, a, o);
                b += __shfl_xor_sync(full, b, o);
            }
            if ((threadIdx.x & 31) == 0) {
                atomicAdd(&sG[j], a);           // W1
                atomicAdd(&sG[kMlpH + j], b);   // b1
            }
        }
        // W2 gradient: sum over the block's samples of dz2[k] h1[j]
#pragma unroll
        for (int j = 0; j < kMlpH; ++j) {
            sH1[threadIdx.x][j] = h1[j];
            sD2[threadIdx.x][j] = z2[j];
        }
        __syncthreads();
#pragma unroll
        for (int c = 0; c < kMlpH * kMlpH / kGradThreads; ++c) {
            const int e2 = threadIdx.x + kGradThreads * c;
            const int k = e2 / kMlpH, j = e2 % kMlpH;
            float acc = 0.0f;
            for (int s = 0; s < kGradThreads; ++s) acc = fmaf(sD2[s][k], sH1[s][j], acc);
            gw2[c] += acc;
        }
        __syncthreads();
    }
#pragma unroll
    for (int c = 0; c < kMlpH * kMlpH / kGradThreads; ++c)
        atomicAdd(&grad[kMlpW2 + threadIdx.x + kGradThreads * c], gw2[c]);
    for (int o = 16; o > 0; o >>= 1) lsum += __shfl_xor_sync(full, lsum, o);
    if ((threadIdx.x & 31) == 0) atomicAdd(&sLoss, lsum);
    __syncthreads();
    for (int k = threadIdx.x; k < kMlpH; k += blockDim.x) {
        atomicAdd(&grad[kMlpW1 + k], sG[k]);
        atomicAdd(&grad[kMlpB1 + k], sG[kMlpH + k]);
        atomicAdd(&grad[kMlpB2 + k], sG[2 * kMlpH + k]);
        atomicAdd(&grad[kMlpW3 + k], sG[3 * kMlpH + k]);
    }
    if (threadIdx.x == 0) {
        atomicAdd(&grad[kMlpB3], sG[4 * kMlpH]);
        if (loss) atomicAdd(loss, sLoss);
    }
}

// Adam update of every parameter from grad, then grad = 0.
__global__ void k_mlp_adam(float* __restrict__ p, float* __restrict__ m, float* __restrict__ v,
                           float* __restrict__ grad, float lr, float beta1, float beta2, float eps,
                           float inv_bc1, float inv_bc2) {
    for (int k = blockIdx.x * blockDim.x + threadIdx.x; k < kMlpParams; k += gridDim.x * blockDim.x) {
        const float g = grad[k];
        const float mk = fmaf(beta1, m[k], (1.0f - beta1) * g);
        const float vk = fmaf(beta2, v[k], (1.0f - beta2) * g * g);
        m[k] = mk;
        v[k] = vk;
        p[k] -= lr * (mk * inv_bc1) / (sqrtf(vk * inv_bc2) + eps);
        grad[k] = 0.0f;
    }
}

static int grad_blocks(long long batch) {
    long long b = (batch + kGradThreads - 1) / kGradThreads;
    if (b > 152) b = 152;
    return (int)(b < 1 ? 1 : b);
}

}  // namespace nbc

using namespace nbc;

static bool range_ok(float r_min, float r_max) {
    return std::isfinite(r_min) && std::isfinite(r_max) && r_max > r_min;
}

extern "C" {

size_t nb_mlp_packed_bytes(void) { return sizeof(MlpTC); }

nb_status nb_ewald_factor(const double* r, int64_t n, double beta, double* out, nb_stream stream) {
    if (n < 0 || (n > 0 && (!r || !out)) || !(beta >= 0.0)) return NB_ERR_ARG;
    if (n == 0) return NB_OK;
    long long blocks = (n + 255) / 256;
    if (blocks > 4096) blocks = 4096;
    k_ewald_factor<<<(int)blocks, 256, 0, (cudaStream_t)stream>>>(r, n, beta, out);
    return cudaGetLastError() == cudaSuccess ? NB_OK : NB_ERR_CUDA;
}

nb_status nb_mlp_pack(const float* params, float r_min, float r_max, void* packed, nb_stream stream) {
    if (!params || !packed || !range_ok(r_min, r_max)) return NB_ERR_ARG;
    if ((uintptr_t)packed & 15) return NB_ERR_ARG;
    k_mlp_pack<<<1, 32, 0, (cudaStream_t)stream>>>(params, 0.5f * (r_min + r_max), 2.0f / (r_max - r_min),
                                                   (MlpTC*)packed);
    return cudaGetLastError() == cudaSuccess ? NB_OK : NB_ERR_CUDA;
}

nb_status nb_mlp_forward(const float* params, float r_min, float r_max, const float* r, int64_t n, float* y,
                         nb_stream stream) {
    if (!params || n < 0 || (n > 0 && (!r || !y)) || !range_ok(r_min, r_max)) return NB_ERR_ARG;
    if (n == 0) return NB_OK;
    long long blocks = (n + 255) / 256;
    if (blocks > 4096) blocks = 4096;
    k_mlp_forward<<<(int)blocks, 256, 0, (cudaStream_t)stream>>>(params, 0.5f * (r_min + r_max),
                                                                 2.0f / (r_max - r_min), r, n, y);
    return cudaGetLastError() == cudaSuccess ? NB_OK : NB_ERR_CUDA;
}

nb_status nb_mlp_forward_tc(const void* packed, const float* r, int64_t n, float* y, nb_stream stream) {
    if (!packed || n < 0 || (n > 0 && (!r || !y)) || ((uintptr_t)packed & 15)) return NB_ERR_ARG;
    if (n == 0) return NB_OK;
    long long blocks = ((n + 63) / 64 + 3) / 4;
    if (blocks > 4096) blocks = 4096;
    k_mlp_forward_tc<<<(int)blocks, 128, 0, (cudaStream_t)stream>>>((const MlpTC*)packed, r, n, y);
    return cudaGetLastError() == cudaSuccess ? NB_OK : NB_ERR_CUDA;
}

nb_status nb_mlp_loss_grad(const float* params, float r_min, float r_max, const float* r, const float* t,
                           const float* w, int64_t n, float* grad, float* loss, nb_stream stream) {
    if (!params || !grad || n <= 0 || !r || !t || !range_ok(r_min, r_max)) return NB_ERR_ARG;
    cudaStream_t s = (cudaStream_t)stream;
    if (cudaMemsetAsync(grad, 0, sizeof(float) * kMlpParams, s) != cudaSuccess) return NB_ERR_CUDA;
    if (loss && cudaMemsetAsync(loss, 0, sizeof(float), s) != cudaSuccess) return NB_ERR_CUDA;
    k_mlp_grad<<<grad_blocks(n), kGradThreads, 0, s>>>(params, 0.5f * (r_min + r_max), 2.0f / (r_max - r_min), r,
                                                       t, w, n, 0, n, 1.0f / (float)n, grad, loss);
    return cudaGetLastError() == cudaSuccess ? NB_OK : NB_ERR_CUDA;
}

nb_status nb_mlp_train(float* params, float* state, float r_min, float r_max, const float* r, const float* t,
                       const float* w, int64_t n, int batch, int steps, int step0, int total_steps,
                       float lr_max, float lr_min, float* loss, nb_stream stream) {
    if (!params || !state || !r || !t || n <= 0 || batch <= 0 || steps < 0 || step0 < 0 ||
        total_steps < step0 + steps || !range_ok(r_min, r_max) || !(lr_max > 0.0f) || !(lr_min >= 0.0f))
        return NB_ERR_ARG;
    cudaStream_t s = (cudaStream_t)stream;
    float* m = state;
    float* v = state + kMlpParams;
    float* grad = state + 2 * kMlpParams;
    const float c0 = 0.5f * (r_min + r_max), c1 = 2.0f / (r_max - r_min);
    const double b1 = 0.9, b2 = 0.999;
    if (cudaMemsetAsync(grad, 0, sizeof(float) * kMlpParams, s) != cudaSuccess) return NB_ERR_CUDA;
    if (loss && steps > 0 && cudaMemsetAsync(loss, 0, sizeof(float) * steps, s) != cudaSuccess) return NB_ERR_CUDA;
    for (int i = 0; i < steps; ++i) {
        const int it = step0 + i;   // 0-based step of the whole schedule
        const double lr = lr_min + (lr_max - lr_min) * 0.5 * (1.0 + std::cos(M_PI * it / (double)total_steps));
        const long long start = ((long long)it * batch) % n;
        k_mlp_grad<<<grad_blocks(batch), kGradThreads, 0, s>>>(params, c0, c1, r, t, w, n, start, batch,
                                                               1.0f / (float)batch, grad, loss ? loss + i : nullptr);
        const double bc1 = 1.0 - std::pow(b1, it + 1), bc2 = 1.0 - std::pow(b2, it + 1);
        k_mlp_adam<<<(kMlpParams + 255) / 256, 256, 0, s>>>(params, m, v, grad, (float)lr, (float)b1, (float)b2,
                                                             1e-8f, (float)(1.0 / bc1), (float)(1.0 / bc2));
    }
    return cudaGetLastError() == cudaSuccess ? NB_OK : NB_ERR_CUDA;
}

}  // extern "C"
