// nn_ops.cu - elementwise and reduction kernels of the warm-start network: input
// preparation, 2x2 average pooling and nearest 2x upsampling (and their backward), ReLU
// backward, skip-gradient addition, bias gradients, the offset-invariant phase loss,
// Adam, weight packing and the bilinear phase output. Tensors are channels-last bf16 with
// C a multiple of 8, handled 8 channels (16 bytes) per thread.
#include <cuda_bf16.h>

#include "nn.h"
#include "runtime.h"

namespace holo {
namespace nn {

constexpr int kThreads = 256;

static int blocks_for(size_t n) { return int((n + kThreads - 1) / kThreads); }

__device__ __forceinline__ void unpack8(const uint4& u, float (&f)[8]) {
    const __nv_bfloat162* h = reinterpret_cast<const __nv_bfloat162*>(&u);
#pragma unroll
    for (int i = 0; i < 4; ++i) {
        const float2 t = __bfloat1622float2(h[i]);
        f[2 * i] = t.x;
        f[2 * i + 1] = t.y;
    }
}
__device__ __forceinline__ uint4 pack8(const float (&f)[8]) {
    uint4 u;
    __nv_bfloat162* h = reinterpret_cast<__nv_bfloat162*>(&u);
#pragma unroll
    for (int i = 0; i < 4; ++i) h[i] = __floats2bfloat162_rn(f[2 * i], f[2 * i + 1]);
    return u;
}

// ---------------------------------------------------------------- input ----
__global__ void k_prep_input(const float* __restrict__ t, int B, int Hs, int Ws, int H, int W, int f,
                             __nv_bfloat16* __restrict__ x, int C) {
    const size_t i = size_t(blockIdx.x) * blockDim.x + threadIdx.x;
    if (i >= size_t(B) * H * W) return;
    const int b = int(i / (size_t(H) * W)), rem = int(i % (size_t(H) * W)), y = rem / W, xx = rem % W;
    float s = 0.f;
    for (int dy = 0; dy < f; ++dy)
        for (int dx = 0; dx < f; ++dx) s += t[(size_t(b) * Hs + y * f + dy) * Ws + xx * f + dx];
    s /= float(f * f);
    uint4* o = reinterpret_cast<uint4*>(x + i * C);
    float v[8] = {s, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f};
    o[0] = pack8(v);
    const float z[8] = {0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f};
    for (int k = 1; k < C / 8; ++k) o[k] = pack8(z);
}

int prep_input(const float* target, int B, int Hs, int Ws, int H, int W, __nv_bfloat16* x, int C, cudaStream_t st) {
    if (Hs % H || Ws % W || Hs / H != Ws / W) return fail(HOLO_EINVAL, "prep_input: %dx%d -> %dx%d", Hs, Ws, H, W);
    Launch ln("nn_elementwise", st);
    k_prep_input<<<blocks_for(size_t(B) * H * W), kThreads, 0, st>>>(target, B, Hs, Ws, H, W, Hs / H, x, C);
    return ln.done("prep_input launch");
}

// ------------------------------------------------------------- pooling ----
__global__ void k_avgpool2(const __nv_bfloat16* __restrict__ x, int B, int H, int W, int C,
                           __nv_bfloat16* __restrict__ y) {
    const int G = C / 8, Ho = H / 2, Wo = W / 2;
    const size_t i = size_t(blockIdx.x) * blockDim.x + threadIdx.x;
    if (i >= size_t(B) * Ho * Wo * G) return;
    const int g = int(i % G);
    const size_t q = i / G;
    const int b = int(q / (size_t(Ho) * Wo)), rem = int(q % (size_t(Ho) * Wo)), oy = rem / Wo, ox = rem % Wo;
    float acc[8] = {0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f};
    for (int dy = 0; dy < 2; ++dy)
        for (int dx = 0; dx < 2; ++dx) {
            float f[8];
            unpack8(*reinterpret_cast<const uint4*>(x + ((size_t(b) * H + 2 * oy + dy) * W + 2 * ox + dx) * C + 8 * g), f);
#pragma unroll
            for (int k = 0; k < 8; ++k) acc[k] += f[k];
        }
#pragma unroll
    for (int k = 0; k < 8; ++k) acc[k] *= 0.25f;
    *reinterpret_cast<uint4*>(y + q * C + 8 * g) = pack8(acc);
}

int avgpool2(const __nv_bfloat16* x, int B, int H, int W, int C, __nv_bfloat16* y, cudaStream_t st) {
    Launch ln("nn_elementwise", st);
    k_avgpool2<<<blocks_for(size_t(B) * (H / 2) * (W / 2) * (C / 8)), kThreads, 0, st>>>(x, B, H, W, C, y);
    return ln.done("avgpool2 launch");
}

__global__ void k_avgpool2_bwd(const __nv_bfloat16* __restrict__ dy, int B, int H, int W, int C,
                               __nv_bfloat16* __restrict__ dx, int accumulate) {
    const int G = C / 8, Ho = H / 2, Wo = W / 2;
    const size_t i = size_t(blockIdx.x) * blockDim.x + threadIdx.x;
    if (i >= size_t(B) * H * W * G) return;
    const int g = int(i % G);
    const size_t q = i / G;
    const int b = int(q / (size_t(H) * W)), rem = int(q % (size_t(H) * W)), y = rem / W, x = rem % W;
    float f[8];
    unpack8(*reinterpret_cast<const uint4*>(dy + ((size_t(b) * Ho + y / 2) * Wo + x / 2) * C + 8 * g), f);
    uint4* o = reinterpret_cast<uint4*>(dx + q * C + 8 * g);
    float prev[8] = {0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f};
    if (accumulate) unpack8(*o, prev);
#pragma unroll
    for (int k = 0; k < 8; ++k) f[k] = prev[k] + 0.25f * f[k];
    *o = pack8(f);
}

int avgpool2_bwd(const __nv_bfloat16* dy, int B, int H, int W, int C, __nv_bfloat16* dx, int accumulate,
                 cudaStream_t st) {
    Launch ln("nn_elementwise", st);
    k_avgpool2_bwd<<<blocks_for(size_t(B) * H * W * (C / 8)), kThreads, 0, st>>>(dy, B, H, W, C, dx, accumulate);
    return ln.done("avgpool2_bwd launch");
}

// ----------------------------------------------------------- upsampling ----
__global__ void k_upsample2(const __nv_bfloat16* __restrict__ x, int B, int H, int W, int C,
                            __nv_bfloat16* __restrict__ y) {
    const int G = C / 8, Ho = 2 * H, Wo = 2 * W;
    const size_t i = size_t(blockIdx.x) * blockDim.x + threadIdx.x;
    if (i >= size_t(B) * Ho * Wo * G) return;
    const int g = int(i % G);
    const size_t q = i / G;
    const int b = int(q / (size_t(Ho) * Wo)), rem = int(q % (size_t(Ho) * Wo)), oy = rem / Wo, ox = rem % Wo;
    *reinterpret_cast<uint4*>(y + q * C + 8 * g) =
        *reinterpret_cast<const uint4*>(x + ((size_t(b) * H + oy / 2) * W + ox / 2) * C + 8 * g);
}

int upsample2(const __nv_bfloat16* x, int B, int H, int W, int C, __nv_bfloat16* y, cudaStream_t st) {
    Launch ln("nn_elementwise", st);
    k_upsample2<<<blocks_for(size_t(B) * 4 * H * W * (C / 8)), kThreads, 0, st>>>(x, B, H, W, C, y);
    return ln.done("upsample2 launch");
}

__global__ void k_upsample2_bwd(const __nv_bfloat16* __restrict__ dy, int B, int H, int W, int C,
                                __nv_bfloat16* __restrict__ dx) {
    const int G = C / 8, Wo = 2 * W;
    const size_t i = size_t(blockIdx.x) * blockDim.x + threadIdx.x;
    if (i >= size_t(B) * H * W * G) return;
    const int g = int(i % G);
    const size_t q = i / G;
    const int b = int(q / (size_t(H) * W)), rem = int(q % (size_t(H) * W)), y = rem / W, x = rem % W;
    float acc[8] = {0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f};
    for (int dy2 = 0; dy2 < 2; ++dy2)
        for (int dx2 = 0; dx2 < 2; ++dx2) {
            float f[8];
            unpack8(*reinterpret_cast<const uint4*>(dy + ((size_t(b) * 2 * H + 2 * y + dy2) * Wo + 2 * x + dx2) * C + 8 * g), f);
#pragma unroll
            for (int k = 0; k < 8; ++k) acc[k] += f[k];
        }
    *reinterpret_cast<uint4*>(dx + q * C + 8 * g) = pack8(acc);
}

int upsample2_bwd(const __nv_bfloat16* dy, int B, int H, int W, int C, __nv_bfloat16* dx, cudaStream_t st) {
    Launch ln("nn_elementwise", st);
    k_upsample2_bwd<<<blocks_for(size_t(B) * H * W * (C / 8)), kThreads, 0, st>>>(dy, B, H, W, C, dx);
    return ln.done("upsample2_bwd launch");
}

// ------------------------------------------------------- relu, add, bias ----
__global__ void k_relu_bwd(__nv_bfloat16* __restrict__ d, const __nv_bfloat16* __restrict__ y, size_t n8) {
    const size_t i = size_t(blockIdx.x) * blockDim.x + threadIdx.x;
    if (i >= n8) return;
    float fd[8], fy[8];
    unpack8(reinterpret_cast<const uint4*>(d)[i], fd);
    unpack8(reinterpret_cast<const uint4*>(y)[i], fy);
#pragma unroll
    for (int k = 0; k < 8; ++k) fd[k] = fy[k] > 0.f ? fd[k] : 0.f;
    reinterpret_cast<uint4*>(d)[i] = pack8(fd);
}

int relu_bwd(__nv_bfloat16* d, const __nv_bfloat16* y, size_t n, cudaStream_t st) {
    Launch ln("nn_elementwise", st);
    k_relu_bwd<<<blocks_for(n / 8), kThreads, 0, st>>>(d, y, n / 8);
    return ln.done("relu_bwd launch");
}

__global__ void k_add_inplace(__nv_bfloat16* __restrict__ a, const __nv_bfloat16* __restrict__ b, size_t n8) {
    const size_t i = size_t(blockIdx.x) * blockDim.x + threadIdx.x;
    if (i >= n8) return;
    float fa[8], fb[8];
    unpack8(reinterpret_cast<const uint4*>(a)[i], fa);
    unpack8(reinterpret_cast<const uint4*>(b)[i], fb);
#pragma unroll
    for (int k = 0; k < 8; ++k) fa[k] += fb[k];
    reinterpret_cast<uint4*>(a)[i] = pack8(fa);
}

int add_inplace(__nv_bfloat16* a, const __nv_bfloat16* b, size_t n, cudaStream_t st) {
    Launch ln("nn_elementwise", st);
    k_add_inplace<<<blocks_for(n / 8), kThreads, 0, st>>>(a, b, n / 8);
    return ln.done("add_inplace launch");
}

// each block sums its pixel range for every 8-channel group, then one atomic per channel
__global__ void k_bias_grad(const __nv_bfloat16* __restrict__ g, size_t pixels, int C, float* __restrict__ db,
                            int pix_per_block) {
    extern __shared__ float sb[];
    const int G = C / 8;
    for (int i = threadIdx.x; i < C; i += blockDim.x) sb[i] = 0.f;
    __syncthreads();
    const int lanes_per_pixel = G;
    const int pix_per_iter = blockDim.x / lanes_per_pixel;
    const int gi = threadIdx.x % G, pi = threadIdx.x / G;
    float acc[8] = {0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f};
    if (pi < pix_per_iter) {
        const size_t p0 = size_t(blockIdx.x) * pix_per_block;
        const size_t p1 = p0 + pix_per_block < pixels ? p0 + pix_per_block : pixels;
        for (size_t p = p0 + pi; p < p1; p += pix_per_iter) {
            float f[8];
            unpack8(*reinterpret_cast<const uint4*>(g + p * C + 8 * gi), f);
#pragma unroll
            for (int k = 0; k < 8; ++k) acc[k] += f[k];
        }
#pragma unroll
        for (int k = 0; k < 8; ++k) atomicAdd(&sb[8 * gi + k], acc[k]);
    }
    __syncthreads();
    for (int i = threadIdx.x; i < C; i += blockDim.x) atomicAdd(db + i, sb[i]);
}

int bias_grad(const __nv_bfloat16* g, size_t pixels, int C, float* db, cudaStream_t st) {
    const int ppb = 2048;
    const int blocks = int((pixels + ppb - 1) / ppb);
    Launch ln("nn_elementwise", st);
    k_bias_grad<<<blocks, kThreads, sizeof(float) * C, st>>>(g, pixels, C, db, ppb);
    return ln.done("bias_grad launch");
}

// ------------------------------------------------------------ phase loss ----
// scratch[b*4 + {0,1,2}] = sum w (y . z), sum w (y x z), sum w over sample b, where
// y = (u, v)/|(u, v)|, z = exp(i label), w = target^2
__global__ void k_loss_sums(const float* __restrict__ out, int C, const float* __restrict__ label,
                            const float* __restrict__ target, int B, int HW, float* __restrict__ scratch) {
    __shared__ float s[3][kThreads / 32];
    const int b = blockIdx.y;
    float sr = 0.f, si = 0.f, sw = 0.f;
    for (int p = blockIdx.x * blockDim.x + threadIdx.x; p < HW; p += gridDim.x * blockDim.x) {
        const size_t q = size_t(b) * HW + p;
        const float u = out[q * C], v = out[q * C + 1];
        const float r = sqrtf(u * u + v * v) + 1e-20f;
        float zs, zc;
        sincosf(label[q], &zs, &zc);
        const float w = target[q] * target[q];
        const float a = u / r, bb = v / r;
        sr += w * (a * zc + bb * zs);
        si += w * (bb * zc - a * zs);
        sw += w;
    }
    for (int o = 16; o > 0; o >>= 1) {
        sr += __shfl_down_sync(0xffffffffu, sr, o);
        si += __shfl_down_sync(0xffffffffu, si, o);
        sw += __shfl_down_sync(0xffffffffu, sw, o);
    }
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    if (lane == 0) {
        s[0][warp] = sr;
        s[1][warp] = si;
        s[2][warp] = sw;
    }
    __syncthreads();
    if (threadIdx.x < 3) {
        float t = 0.f;
        for (int w = 0; w < blockDim.x / 32; ++w) t += s[threadIdx.x][w];
        atomicAdd(scratch + 4 * b + threadIdx.x, t);
    }
}

__global__ void k_loss_grad(const float* __restrict__ out, int C, const float* __restrict__ label,
                            const float* __restrict__ target, int B, int HW, const float* __restrict__ scratch,
                            float* __restrict__ loss, __nv_bfloat16* __restrict__ gout) {
    const size_t q = size_t(blockIdx.x) * blockDim.x + threadIdx.x;
    if (q == 0) {
        float L = 0.f;
        for (int b = 0; b < B; ++b) {
            const float Sr = scratch[4 * b], Si = scratch[4 * b + 1], Wt = scratch[4 * b + 2];
            L += 1.f - sqrtf(Sr * Sr + Si * Si) / fmaxf(Wt, 1e-30f);
        }
        *loss = L / float(B);
    }
    if (q >= size_t(B) * HW) return;
    const int b = int(q / HW);
    const float Sr = scratch[4 * b], Si = scratch[4 * b + 1], Wt = scratch[4 * b + 2];
    const float mag = sqrtf(Sr * Sr + Si * Si) + 1e-20f;
    const float u = out[q * C], v = out[q * C + 1];
    const float r = sqrtf(u * u + v * v) + 1e-20f;
    float zs, zc;
    sincosf(label[q], &zs, &zc);
    const float w = target[q] * target[q];
    const float k = -w / (float(B) * fmaxf(Wt, 1e-30f) * mag);
    const float ga = k * (Sr * zc - Si * zs), gb = k * (Sr * zs + Si * zc);
    const float r3 = r * r * r;
    const float gu = v * (ga * v - gb * u) / r3, gv = u * (gb * u - ga * v) / r3;
    float f[8] = {gu, gv, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f};
    uint4* o = reinterpret_cast<uint4*>(gout + q * C);
    o[0] = pack8(f);
    const float z[8] = {0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f};
    for (int g = 1; g < C / 8; ++g) o[g] = pack8(z);
}

int phase_loss(const float* out, int C, const float* label, const float* target, int B, int HW, float* scratch,
               float* loss, __nv_bfloat16* gout, cudaStream_t st) {
    int rc = cuda_status(cudaMemsetAsync(scratch, 0, sizeof(float) * 4 * B, st), "phase_loss: reset");
    if (rc) return rc;
    {
        Launch ln("nn_loss", st);
        dim3 grid(64, B);
        k_loss_sums<<<grid, kThreads, 0, st>>>(out, C, label, target, B, HW, scratch);
        if ((rc = ln.done("loss_sums launch"))) return rc;
    }
    Launch ln("nn_loss", st);
    k_loss_grad<<<blocks_for(size_t(B) * HW), kThreads, 0, st>>>(out, C, label, target, B, HW, scratch, loss, gout);
    return ln.done("loss_grad launch");
}

// ------------------------------------------------------------------ adam ----
__global__ void k_adam(float* __restrict__ w, const float* __restrict__ g, float* __restrict__ m,
                       float* __restrict__ v, size_t n, float lr, float b1, float b2, float eps, float c1, float c2) {
    const size_t i = size_t(blockIdx.x) * blockDim.x + threadIdx.x;
    if (i >= n) return;
    const float gi = g[i];
    const float mi = b1 * m[i] + (1.f - b1) * gi;
    const float vi = b2 * v[i] + (1.f - b2) * gi * gi;
    m[i] = mi;
    v[i] = vi;
    w[i] -= lr * (mi / c1) / (sqrtf(vi / c2) + eps);
}

int adam(float* w, const float* g, float* m, float* v, size_t n, float lr, float b1, float b2, float eps, int step,
         cudaStream_t st) {
    const float c1 = 1.f - powf(b1, float(step)), c2 = 1.f - powf(b2, float(step));
    Launch ln("nn_adam", st);
    k_adam<<<blocks_for(n), kThreads, 0, st>>>(w, g, m, v, n, lr, b1, b2, eps, c1, c2);
    return ln.done("adam launch");
}

__global__ void k_pack_weights(const float* __restrict__ w, int Cout, int Cin, __nv_bfloat16* __restrict__ wmat,
                               __nv_bfloat16* __restrict__ wt) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= Cout * 9 * Cin) return;
    const int co = i / (9 * Cin), rem = i % (9 * Cin), tap = rem / Cin, ci = rem % Cin;
    const __nv_bfloat16 h = __float2bfloat16_rn(w[i]);
    wmat[i] = h;
    wt[(size_t(ci) * 9 + tap) * Cout + co] = h;
}

int pack_weights(const float* w, int Cout, int Cin, __nv_bfloat16* wmat, __nv_bfloat16* wt, cudaStream_t st) {
    Launch ln("nn_elementwise", st);
    k_pack_weights<<<blocks_for(size_t(Cout) * 9 * Cin), kThreads, 0, st>>>(w, Cout, Cin, wmat, wt);
    return ln.done("pack_weights launch");
}

// --------------------------------------------------------------- output ----
// Sample position of output index o (of n_out) on an input axis of n_in pixels, half-pixel
// centres: s = (o + 1/2) n_in / n_out - 1/2 = ((2o + 1) n_in - n_out) / (2 n_out), clamped
// to [0, n_in - 1]. The neighbour i0 = floor(s) is exact (integer division) and the
// fraction f = s - i0 is one float division of exact integers.
__device__ __forceinline__ void sample_axis(int o, int n_in, int n_out, int& i0, int& i1, float& f) {
    const int64_t num = (2 * int64_t(o) + 1) * n_in - n_out;
    const int64_t den = 2 * int64_t(n_out);
    if (num <= 0) {
        i0 = 0;
        f = 0.f;
    } else {
        const int64_t q = num / den;
        if (q >= n_in - 1) {
            i0 = n_in - 1;
            f = 0.f;
        } else {
            i0 = int(q);
            f = float(num - q * den) / float(den);
        }
    }
    i1 = i0 + 1 < n_in ? i0 + 1 : i0;
}

__global__ void k_phase_out(const float* __restrict__ out, int C, int H, int W, int Ho, int Wo,
                            float* __restrict__ phase) {
    const size_t i = size_t(blockIdx.x) * blockDim.x + threadIdx.x;
    if (i >= size_t(Ho) * Wo) return;
    const int oy = int(i / Wo), ox = int(i % Wo);
    int y0, y1, x0, x1;
    float fy, fx;
    sample_axis(oy, H, Ho, y0, y1, fy);
    sample_axis(ox, W, Wo, x0, x1, fx);
    float u = 0.f, v = 0.f;
    const int ys[2] = {y0, y1}, xs[2] = {x0, x1};
    const float wy[2] = {1.f - fy, fy}, wx[2] = {1.f - fx, fx};
    for (int a = 0; a < 2; ++a)
        for (int b = 0; b < 2; ++b) {
            const size_t q = (size_t(ys[a]) * W + xs[b]) * C;
            u += wy[a] * wx[b] * out[q];
            v += wy[a] * wx[b] * out[q + 1];
        }
    phase[i] = atan2f(v, u);
}

int phase_out(const float* out, int C, int H, int W, int Ho, int Wo, float* phase, cudaStream_t st) {
    Launch ln("nn_elementwise", st);
    k_phase_out<<<blocks_for(size_t(Ho) * Wo), kThreads, 0, st>>>(out, C, H, W, Ho, Wo, phase);
    return ln.done("phase_out launch");
}

}  // namespace nn
}  // namespace holo
