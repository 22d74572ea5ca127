// nn_conv.cu - 3x3 convolution (zero padding 1, stride 1) of the warm-start network as an
// implicit GEMM on the tensor cores: bf16 operands, float32 accumulation
// (mma.sync.m16n8k16). Activations are channels-last [B][H][W][C] bf16 with C a multiple
// of 8; weights are [Cout][3][3][Cin] (a row-major [Cout][9*Cin] matrix).
//
//   forward  Y[p][o] = act(sum_k X(p, k) Wm[o][k] + bias[o] + R[p][o])   M = pixels, N = Cout,
//            k = 9*Cin, X(p, (tap, i)) = x[b][y+ky-1][x+kx-1][i] (0 outside)
//   dgrad    dX[p][i] = sum_k dY(p, k) Wt[i][k], k = (tap, o), dY(p, (tap, o)) =
//            dy[b][y+1-ky][x+1-kx][o], Wt[i][tap][o] = W[o][tap][i]    (same kernel, flipped)
//   wgrad    dW[o][(tap, i)] += sum_p dy[p][o] X(p, (tap, i))            M = Cout, N = 9*Cin,
//            K = pixels, split over blockIdx.z and accumulated with float atomics
// The GEMM operands are gathered on the fly from the activations (no im2col buffer).
#include <cuda_bf16.h>

#include "nn.h"
#include "runtime.h"

namespace holo {
namespace nn {

constexpr int BM = 64, BN = 64, BK = 32, KP = BK + 8;   // KP: padded smem row (bank spread)

__device__ __forceinline__ void mma_bf16_16816(float (&d)[4], const uint32_t (&a)[4], uint32_t b0, uint32_t b1) {
    asm volatile(
        "mma.sync.aligned.m16n8k16.row.col.f32.bf16.bf16.f32 {%0,%1,%2,%3}, {%4,%5,%6,%7}, {%8,%9}, "
        "{%0,%1,%2,%3};\n"
        : "+f"(d[0]), "+f"(d[1]), "+f"(d[2]), "+f"(d[3])
        : "r"(a[0]), "r"(a[1]), "r"(a[2]), "r"(a[3]), "r"(b0), "r"(b1));
}

// 8 consecutive channels of pixel (b, y, x) of a [B][H][W][C] tensor, zero outside
__device__ __forceinline__ uint4 load8(const __nv_bfloat16* t, int b, int y, int x, int c, int H, int W, int C) {
    if (y < 0 || y >= H || x < 0 || x >= W) return make_uint4(0u, 0u, 0u, 0u);
    return *reinterpret_cast<const uint4*>(t + ((size_t(b) * H + y) * W + x) * C + c);
}

template <int MODE>
__global__ void __launch_bounds__(128) k_conv3x3(ConvArgs a) {
    __shared__ __align__(16) __nv_bfloat16 As[BM][KP];
    __shared__ __align__(16) __nv_bfloat16 Bs[BN][KP];
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const int wm = warp >> 1, wn = warp & 1;
    const int g = lane >> 2, c = lane & 3;
    const int HW = a.H * a.W;
    int M, N, K;
    if (MODE == kConvWgrad) {
        M = a.Cout; N = 9 * a.Cin; K = a.B * HW;
    } else {
        M = a.B * HW; N = a.Cout; K = 9 * a.Cin;
    }
    const int m0 = blockIdx.y * BM, n0 = blockIdx.x * BN;
    int kbeg = 0, kend = K;
    if (MODE == kConvWgrad) {
        kbeg = blockIdx.z * a.kchunk;
        kend = min(K, kbeg + a.kchunk);
    }
    float acc[2][4][4];
#pragma unroll
    for (int i = 0; i < 2; ++i)
#pragma unroll
        for (int j = 0; j < 4; ++j)
#pragma unroll
            for (int q = 0; q < 4; ++q) acc[i][j][q] = 0.f;

    for (int k0 = kbeg; k0 < kend; k0 += BK) {
        if (MODE != kConvWgrad) {
#pragma unroll
            for (int i = 0; i < 2; ++i) {
                const int idx = tid + 128 * i;
                const int row = idx >> 2, kv = (idx & 3) * 8;
                const int k = k0 + kv;
                uint4 xv = make_uint4(0u, 0u, 0u, 0u);
                const int m = m0 + row;
                if (m < M && k < kend) {
                    const int tap = k / a.Cin, ci = k - tap * a.Cin;
                    const int ky = tap / 3, kx = tap - 3 * ky;
                    const int b = m / HW, rem = m - b * HW, y = rem / a.W, x = rem - y * a.W;
                    const int yy = a.flip ? y + 1 - ky : y + ky - 1;
                    const int xx = a.flip ? x + 1 - kx : x + kx - 1;
                    xv = load8(a.in, b, yy, xx, ci, a.H, a.W, a.Cin);
                }
                *reinterpret_cast<uint4*>(&As[row][kv]) = xv;
                const int n = n0 + row;
                uint4 wv = make_uint4(0u, 0u, 0u, 0u);
                if (n < N && k < kend) wv = *reinterpret_cast<const uint4*>(a.wmat + size_t(n) * K + k);
                *reinterpret_cast<uint4*>(&Bs[row][kv]) = wv;
            }
        } else {
#pragma unroll
            for (int i = 0; i < 2; ++i) {
                const int idx = tid + 128 * i;
                const int pl = idx >> 3, cv = (idx & 7) * 8;
                const int p = k0 + pl;
                uint4 dv = make_uint4(0u, 0u, 0u, 0u), xv = make_uint4(0u, 0u, 0u, 0u);
                if (p < kend) {
                    if (m0 + cv < M) dv = *reinterpret_cast<const uint4*>(a.dy + size_t(p) * a.Cout + m0 + cv);
                    const int n = n0 + cv;
                    if (n < N) {
                        const int tap = n / a.Cin, ci = n - tap * a.Cin;
                        const int ky = tap / 3, kx = tap - 3 * ky;
                        const int b = p / HW, rem = p - b * HW, y = rem / a.W, x = rem - y * a.W;
                        xv = load8(a.in, b, y + ky - 1, x + kx - 1, ci, a.H, a.W, a.Cin);
                    }
                }
                const __nv_bfloat16* d8 = reinterpret_cast<const __nv_bfloat16*>(&dv);
                const __nv_bfloat16* x8 = reinterpret_cast<const __nv_bfloat16*>(&xv);
#pragma unroll
                for (int j = 0; j < 8; ++j) {
                    As[cv + j][pl] = d8[j];
                    Bs[cv + j][pl] = x8[j];
                }
            }
        }
        __syncthreads();
#pragma unroll
        for (int kk = 0; kk < BK; kk += 16) {
            uint32_t af[2][4], bf[4][2];
#pragma unroll
            for (int mt = 0; mt < 2; ++mt) {
                const int r = wm * 32 + mt * 16 + g;
                af[mt][0] = *reinterpret_cast<const uint32_t*>(&As[r][kk + 2 * c]);
                af[mt][1] = *reinterpret_cast<const uint32_t*>(&As[r + 8][kk + 2 * c]);
                af[mt][2] = *reinterpret_cast<const uint32_t*>(&As[r][kk + 2 * c + 8]);
                af[mt][3] = *reinterpret_cast<const uint32_t*>(&As[r + 8][kk + 2 * c + 8]);
            }
#pragma unroll
            for (int nt = 0; nt < 4; ++nt) {
                const int col = wn * 32 + nt * 8 + g;
                bf[nt][0] = *reinterpret_cast<const uint32_t*>(&Bs[col][kk + 2 * c]);
                bf[nt][1] = *reinterpret_cast<const uint32_t*>(&Bs[col][kk + 2 * c + 8]);
            }
#pragma unroll
            for (int mt = 0; mt < 2; ++mt)
#pragma unroll
                for (int nt = 0; nt < 4; ++nt) mma_bf16_16816(acc[mt][nt], af[mt], bf[nt][0], bf[nt][1]);
        }
        __syncthreads();
    }

#pragma unroll
    for (int mt = 0; mt < 2; ++mt)
#pragma unroll
        for (int nt = 0; nt < 4; ++nt)
#pragma unroll
            for (int h = 0; h < 2; ++h) {
                const int row = m0 + wm * 32 + mt * 16 + g + 8 * h;
                const int col = n0 + wn * 32 + nt * 8 + 2 * c;
                if (row >= M || col >= N) continue;
                float v0 = acc[mt][nt][2 * h], v1 = acc[mt][nt][2 * h + 1];
                if (MODE == kConvWgrad) {
                    atomicAdd(a.dw + size_t(row) * N + col, v0);
                    if (col + 1 < N) atomicAdd(a.dw + size_t(row) * N + col + 1, v1);
                } else {
                    const size_t o = size_t(row) * N + col;
                    if (a.bias) {
                        v0 += a.bias[col];
                        v1 += a.bias[col + 1];
                    }
                    if (a.residual) {
                        const float2 r2 = __bfloat1622float2(*reinterpret_cast<const __nv_bfloat162*>(a.residual + o));
                        v0 += r2.x;
                        v1 += r2.y;
                    }
                    if (a.relu) {
                        v0 = fmaxf(v0, 0.f);
                        v1 = fmaxf(v1, 0.f);
                    }
                    if (a.out) *reinterpret_cast<__nv_bfloat162*>(a.out + o) = __floats2bfloat162_rn(v0, v1);
                    if (a.out_f32) *reinterpret_cast<float2*>(a.out_f32 + o) = make_float2(v0, v1);
                }
            }
}

int conv3x3(const ConvArgs& a, int mode, cudaStream_t st, bool legacy) {
    if (a.Cin % 8 || a.Cout % 8) return fail(HOLO_EINVAL, "conv3x3: channels must be multiples of 8");
    if (mode != kConvWgrad && !legacy && conv3x3_tc05_supported(a)) return conv3x3_tc05(a, mode, st);
    const int P = a.B * a.H * a.W;
    if (mode == kConvWgrad) {
        ConvArgs b = a;
        const int M = a.Cout, N = 9 * a.Cin;
        // split the pixel reduction so that the grid fills the GPU
        const int tiles = ((N + BN - 1) / BN) * ((M + BM - 1) / BM);
        int splits = (2 * 152 + tiles - 1) / tiles;
        int chunk = ((P + splits - 1) / splits + BK - 1) / BK * BK;
        if (chunk < BK) chunk = BK;
        splits = (P + chunk - 1) / chunk;
        b.kchunk = chunk;
        dim3 grid((N + BN - 1) / BN, (M + BM - 1) / BM, splits);
        Launch ln("nn_conv_wgrad", st);
        k_conv3x3<kConvWgrad><<<grid, 128, 0, st>>>(b);
        return ln.done("nn_conv_wgrad launch");
    }
    dim3 grid((a.Cout + BN - 1) / BN, (P + BM - 1) / BM, 1);
    Launch ln(mode == kConvFwd ? "nn_conv_fwd" : "nn_conv_dgrad", st);
    k_conv3x3<kConvFwd><<<grid, 128, 0, st>>>(a);
    return ln.done("nn_conv launch");
}

}  // namespace nn
}  // namespace holo
