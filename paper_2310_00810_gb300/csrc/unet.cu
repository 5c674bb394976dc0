// Learned inlet-profile initialiser (include/unet.h): a 4-level U-Net,
// forward and backward, BF16 operands with FP32 accumulation on the tensor
// cores (mma.sync m16n8k16), FP32 master weights and Adam.
//
// Every convolution is an implicit GEMM through one kernel, k_gemm, whose
// operand loaders and epilogue are template parameters:
//   3x3 convolution        C[pixel][co]  = sum_(tap,ci) X[pixel+tap][ci]  W[tap][ci][co]      (+bias, ReLU)
//   its input gradient     C[pixel][ci]  = sum_(tap,co) G[pixel-tap][co]  W[tap][ci][co]
//                          (the same GEMM with the taps flipped and the channel roles swapped)
//   its weight gradient    C[(tap,ci)][co] = sum_pixel X[pixel+tap][ci] G[pixel][co]          (split-K)
//   2x2 stride-2 transposed convolution: one GEMM per output phase (dy, dx), and its two
//   gradients the same way.
// A CTA computes a 128 x 64 tile of C with 8 warps (32 x 32 each), staging
// 128 x 32 and 64 x 32 operand tiles in shared memory (k contiguous, rows
// padded to 40 elements: conflict-free fragment loads).  Activations are
// NHWC bf16 with channel counts that are multiples of 8, so every operand
// load is a 16-byte vector.  Weight-gradient GEMMs split the pixel sum over
// blockIdx.z into FP32 partials that a second kernel adds in a fixed order
// (deterministic), as are the bias and head reductions.
#include <cuda_bf16.h>

#include <algorithm>
#include <type_traits>
#include <vector>

#include "../../include/unet.h"
#include "common.cuh"
#include "umma.cuh"

namespace lbm {
namespace {

using bf16 = __nv_bfloat16;

constexpr int BM = 128, BN = 64, BK = 32, LDS = BK + 8;
constexpr int kGemmThreads = 256;

__device__ __forceinline__ void mma16816(float (&c)[4], const uint32_t (&a)[4], const uint32_t (&b)[2])
{
    asm volatile(
        "mma.sync.aligned.m16n8k16.row.col.f32.bf16.bf16.f32 {%0,%1,%2,%3}, {%4,%5,%6,%7}, {%8,%9}, "
        "{%0,%1,%2,%3};"
        : "+f"(c[0]), "+f"(c[1]), "+f"(c[2]), "+f"(c[3])
        : "r"(a[0]), "r"(a[1]), "r"(a[2]), "r"(a[3]), "r"(b[0]), "r"(b[1]));
}

// Four 8x8 b16 matrices from shared memory, transposed: thread t receives,
// of matrix q (row addresses from threads 8q..8q+7), the elements
// (row 2 (t % 4), column t / 4) and (row 2 (t % 4) + 1, column t / 4).
__device__ __forceinline__ void ldmatrix_x4_trans(uint32_t (&r)[4], const void* row_addr)
{
    asm volatile("ldmatrix.sync.aligned.m8n8.x4.trans.shared.b16 {%0,%1,%2,%3}, [%4];"
                 : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3])
                 : "r"((uint32_t)__cvta_generic_to_shared(row_addr)));
}

// The same without transposition: thread t receives, of matrix q, the
// elements (row t / 4, columns 2 (t % 4) and 2 (t % 4) + 1).
__device__ __forceinline__ void ldmatrix_x4(uint32_t (&r)[4], const void* row_addr)
{
    asm volatile("ldmatrix.sync.aligned.m8n8.x4.shared.b16 {%0,%1,%2,%3}, [%4];"
                 : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3])
                 : "r"((uint32_t)__cvta_generic_to_shared(row_addr)));
}

// Pixel (b, y, x) of an image batch [b][h][w].
struct Pix {
    int b, y, x;
};

// ---------------------------------------------------------------- loaders
// Each stages a ROWS x BK operand tile (row index = m or n, k contiguous) in
// three steps: prepare(r0) once per CTA (the per-thread row coordinates,
// fixed along k), fetch(k0, kend) global -> registers (zeros outside
// [0, R) x [k0, kend)), put(S) registers -> shared memory.  fetch of the next
// tile is issued before the MMAs of the current one.  Pixel counts stay below
// 2^31, so index arithmetic is 32-bit except the final address.

template <int ROWS>
struct Items {
    static constexpr int N = ROWS * (BK / 8) / kGemmThreads;  // 16-byte items per thread
};

// Rows of an activation batch gathered through a tap (3x3 with zero padding,
// or 1 tap): row = pixel, k = tap * C + c.
template <int ROWS>
struct LdIm2col {
    static constexpr bool KMAJOR = false;  // shared tile [row][k]
    const bf16* x;
    int H, W, C, ld, off, taps;
    static constexpr int NI = Items<ROWS>::N;
    int y[NI], xw[NI];
    size_t base[NI];
    bool ok[NI];
    uint4 v[NI];
    __device__ void set_phase(int) {}
    __device__ void prepare(long long r0, long long R)
    {
#pragma unroll
        for (int i = 0; i < NI; ++i) {
            const int e = threadIdx.x + i * kGemmThreads, r = e >> 2;
            const long long m = r0 + r;
            ok[i] = m < R;
            const int mi = ok[i] ? (int)m : 0;
            xw[i] = mi % W;
            const int t = mi / W;
            y[i] = t % H;
            base[i] = ((size_t)(t / H) * H * W + (size_t)y[i] * W + xw[i]) * ld + off;
        }
    }
    __device__ void fetch(int k0, int kend)
    {
#pragma unroll
        for (int i = 0; i < NI; ++i) {
            const int e = threadIdx.x + i * kGemmThreads, j = e & 3;
            const int k = k0 + 8 * j;
            v[i] = make_uint4(0, 0, 0, 0);
            if (ok[i] && k < kend) {
                const int tap = k / C, ci = k - tap * C;
                const int dy = taps == 9 ? tap / 3 - 1 : 0, dx = taps == 9 ? tap % 3 - 1 : 0;
                const int yy = y[i] + dy, xx = xw[i] + dx;
                if (yy >= 0 && yy < H && xx >= 0 && xx < W)
                    v[i] = *reinterpret_cast<const uint4*>(x + base[i] + (long long)(dy * W + dx) * ld + ci);
            }
        }
    }
    __device__ void put(bf16 (*S)[LDS]) const
    {
#pragma unroll
        for (int i = 0; i < NI; ++i) {
            const int e = threadIdx.x + i * kGemmThreads;
            *reinterpret_cast<uint4*>(&S[e >> 2][8 * (e & 3)]) = v[i];
        }
    }
};

// The gradient of a 2x2 stride-2 transposed convolution's output, gathered
// onto its input pixels: row = input pixel (b, y, x) of an H x W image,
// k = phase * C + c, value dY[b][2y + dy][2x + dx][c].
template <int ROWS>
struct LdUpGather {
    static constexpr bool KMAJOR = false;  // shared tile [row][k]
    const bf16* g;
    int H, W, C, ld, off;
    static constexpr int NI = Items<ROWS>::N;
    size_t base[NI];
    bool ok[NI];
    uint4 v[NI];
    __device__ void set_phase(int) {}
    __device__ void prepare(long long r0, long long R)
    {
#pragma unroll
        for (int i = 0; i < NI; ++i) {
            const int e = threadIdx.x + i * kGemmThreads;
            const long long m = r0 + (e >> 2);
            ok[i] = m < R;
            const int mi = ok[i] ? (int)m : 0;
            const int x = mi % W, t = mi / W, y = t % H, b = t / H;
            base[i] = (((size_t)b * 2 * H + 2 * y) * (2 * W) + 2 * x) * ld + off;
        }
    }
    __device__ void fetch(int k0, int kend)
    {
#pragma unroll
        for (int i = 0; i < NI; ++i) {
            const int e = threadIdx.x + i * kGemmThreads, k = k0 + 8 * (e & 3);
            v[i] = make_uint4(0, 0, 0, 0);
            if (ok[i] && k < kend) {
                const int ph = k / C, c = k - ph * C;
                v[i] = *reinterpret_cast<const uint4*>(g + base[i] + (long long)((ph >> 1) * 2 * W + (ph & 1)) * ld + c);
            }
        }
    }
    __device__ void put(bf16 (*S)[LDS]) const
    {
#pragma unroll
        for (int i = 0; i < NI; ++i) {
            const int e = threadIdx.x + i * kGemmThreads;
            *reinterpret_cast<uint4*>(&S[e >> 2][8 * (e & 3)]) = v[i];
        }
    }
};

// Weight rows: S[r][k] = w[row * ld + k] (+ phase * phase_stride).
template <int ROWS>
struct LdRows {
    static constexpr bool KMAJOR = false;  // shared tile [row][k]
    const bf16* w;
    int ld;
    long long phase_stride;
    static constexpr int NI = Items<ROWS>::N;
    size_t base[NI];
    bool ok[NI];
    uint4 v[NI];
    __device__ void set_phase(int ph) { w += ph * phase_stride; }
    __device__ void prepare(long long r0, long long R)
    {
#pragma unroll
        for (int i = 0; i < NI; ++i) {
            const long long n = r0 + ((threadIdx.x + i * kGemmThreads) >> 2);
            ok[i] = n < R;
            base[i] = ok[i] ? (size_t)n * ld : 0;
        }
    }
    __device__ void fetch(int k0, int kend)
    {
#pragma unroll
        for (int i = 0; i < NI; ++i) {
            const int k = k0 + 8 * ((threadIdx.x + i * kGemmThreads) & 3);
            v[i] = ok[i] && k < kend ? *reinterpret_cast<const uint4*>(w + base[i] + k) : make_uint4(0, 0, 0, 0);
        }
    }
    __device__ void put(bf16 (*S)[LDS]) const
    {
#pragma unroll
        for (int i = 0; i < NI; ++i) {
            const int e = threadIdx.x + i * kGemmThreads;
            *reinterpret_cast<uint4*>(&S[e >> 2][8 * (e & 3)]) = v[i];
        }
    }
};

// Transposed gather for weight gradients: row = (tap, c) with tap in
// [0, taps), k = pixel; value X[pixel + tap][c] (zero padding).  With up = 1
// the pixel is an input pixel of a transposed convolution and the value comes
// from its output pixel (2y + dy, 2x + dx) of the 2H x 2W image (phase from
// set_phase).
template <int ROWS>
struct LdGatherT {
    static constexpr bool KMAJOR = true;  // shared tile [k][row]: fragments through ldmatrix.trans
    const bf16* x;
    int H, W, C, ld, off, taps;
    int up;
    int ph;
    static constexpr int CH = ROWS / 8;                     // 8-row chunks per k
    static constexpr int NI = BK * CH / kGemmThreads;       // items per thread
    int dy[NI], dx[NI], c[NI];
    bool ok[NI];
    uint4 v[NI];
    __device__ void set_phase(int p) { ph = p; }
    __device__ void prepare(long long r0, long long R)
    {
#pragma unroll
        for (int i = 0; i < NI; ++i) {
            const int e = threadIdx.x + i * kGemmThreads, jc = e % CH;
            const long long m = r0 + 8 * jc;
            ok[i] = m < R;
            const int mi = ok[i] ? (int)m : 0;
            const int tap = mi / C;
            c[i] = mi - tap * C;
            dy[i] = up ? ph >> 1 : (taps == 9 ? tap / 3 - 1 : 0);
            dx[i] = up ? ph & 1 : (taps == 9 ? tap % 3 - 1 : 0);
        }
    }
    __device__ void fetch(int k0, int kend)
    {
#pragma unroll
        for (int i = 0; i < NI; ++i) {
            const int e = threadIdx.x + i * kGemmThreads, kk = e / CH;
            const int k = k0 + kk;
            v[i] = make_uint4(0, 0, 0, 0);
            if (ok[i] && k < kend) {
                const int xw = k % W, t = k / W, y = t % H, b = t / H;
                if (up) {
                    const size_t a = (((size_t)b * 2 * H + 2 * y + dy[i]) * (2 * W) + 2 * xw + dx[i]) * ld + off + c[i];
                    v[i] = *reinterpret_cast<const uint4*>(x + a);
                } else {
                    const int yy = y + dy[i], xx = xw + dx[i];
                    if (yy >= 0 && yy < H && xx >= 0 && xx < W)
                        v[i] = *reinterpret_cast<const uint4*>(x + (((size_t)b * H + yy) * W + xx) * ld + off + c[i]);
                }
            }
        }
    }
    __device__ void put(bf16 (*S)[ROWS + 8]) const
    {
#pragma unroll
        for (int i = 0; i < NI; ++i) {
            const int e = threadIdx.x + i * kGemmThreads, kk = e / CH, jc = e % CH;
            *reinterpret_cast<uint4*>(&S[kk][8 * jc]) = v[i];
        }
    }
};

// -------------------------------------------------------------- epilogues

// y[m][off + n] = act(acc + bias[n]) in bf16.
struct EpAct {
    bf16* y;
    int ld, off;
    const float* bias;
    int relu;
    __device__ void set_phase(int) {}
    __device__ void store(long long m, int n, float v0, float v1) const
    {
        if (bias) {
            v0 += bias[n];
            v1 += bias[n + 1];
        }
        if (relu) {
            v0 = fmaxf(v0, 0.0f);
            v1 = fmaxf(v1, 0.0f);
        }
        *reinterpret_cast<__nv_bfloat162*>(y + (size_t)m * ld + off + n) = __floats2bfloat162_rn(v0, v1);
    }
    // eight consecutive columns n .. n + 7 (n a multiple of 8): one 16-byte store
    __device__ void store8(long long m, int n, const float (&v)[8]) const
    {
        union {
            uint4 u;
            __nv_bfloat162 h[4];
        } o;
#pragma unroll
        for (int j = 0; j < 4; ++j) {
            float a = v[2 * j], b = v[2 * j + 1];
            if (bias) {
                a += bias[n + 2 * j];
                b += bias[n + 2 * j + 1];
            }
            if (relu) {
                a = fmaxf(a, 0.0f);
                b = fmaxf(b, 0.0f);
            }
            o.h[j] = __floats2bfloat162_rn(a, b);
        }
        *reinterpret_cast<uint4*>(y + (size_t)m * ld + off + n) = o.u;
    }
};

// Transposed-convolution output: input pixel m of an H x W image -> output
// pixel (2y + dy, 2x + dx) of the 2H x 2W image, + bias, no activation.
struct EpUp {
    bf16* y;
    int H, W, ld, off;
    const float* bias;
    int ph;
    __device__ void set_phase(int p) { ph = p; }
    __device__ void store(long long m, int n, float v0, float v1) const
    {
        const int mi = (int)m, x = mi % W, t = mi / W;
        const Pix p{t / H, t % H, x};
        const int yy = 2 * p.y + ph / 2, xx = 2 * p.x + ph % 2;
        v0 += bias[n];
        v1 += bias[n + 1];
        *reinterpret_cast<__nv_bfloat162*>(y + ((size_t)((long long)p.b * 2 * H + yy) * (2 * W) + xx) * ld + off + n) =
            __floats2bfloat162_rn(v0, v1);
    }
    __device__ void store8(long long m, int n, const float (&v)[8]) const
    {
        const int mi = (int)m, x = mi % W, t = mi / W;
        const Pix p{t / H, t % H, x};
        const int yy = 2 * p.y + ph / 2, xx = 2 * p.x + ph % 2;
        union {
            uint4 u;
            __nv_bfloat162 h[4];
        } o;
#pragma unroll
        for (int j = 0; j < 4; ++j) o.h[j] = __floats2bfloat162_rn(v[2 * j] + bias[n + 2 * j], v[2 * j + 1] + bias[n + 2 * j + 1]);
        *reinterpret_cast<uint4*>(y + ((size_t)((long long)p.b * 2 * H + yy) * (2 * W) + xx) * ld + off + n) = o.u;
    }
};

// FP32 partial of a split-K product: p[split][phase][m][n].
struct EpPartial {
    float* p;
    int N;
    long long split_stride, phase_stride;
    int split, ph;
    __device__ void set_phase(int q) { ph = q; }
    __device__ void store(long long m, int n, float v0, float v1) const
    {
        float* d = p + split * split_stride + ph * phase_stride + m * N + n;
        d[0] = v0;
        d[1] = v1;
    }
    __device__ void store8(long long m, int n, const float (&v)[8]) const
    {
        float4* d = reinterpret_cast<float4*>(p + split * split_stride + ph * phase_stride + m * N + n);
        d[0] = make_float4(v[0], v[1], v[2], v[3]);
        d[1] = make_float4(v[4], v[5], v[6], v[7]);
    }
};

// C[M][N] = sum_k A[m][k] B[n][k] over the k range of split blockIdx.z % splits;
// blockIdx.z / splits is the phase handed to the loaders and the epilogue.
template <class LA, class LB, class EP>
__global__ void __launch_bounds__(kGemmThreads) k_gemm(LA la, LB lb, EP ep, long long M, int N, int K, int k_split,
                                                       int splits)
{
    // operand tiles: [row][k] (k contiguous), or [k][row] for k-major loaders
    constexpr int A_BYTES = (LA::KMAJOR ? BK * (BM + 8) : BM * LDS) * 2;
    constexpr int B_BYTES = (LB::KMAJOR ? BK * (BN + 8) : BN * LDS) * 2;
    __shared__ __align__(16) unsigned char sm[A_BYTES + B_BYTES];
    auto As = reinterpret_cast<bf16(*)[LDS]>(sm);
    auto AsT = reinterpret_cast<bf16(*)[BM + 8]>(sm);
    auto Bs = reinterpret_cast<bf16(*)[LDS]>(sm + A_BYTES);
    auto BsT = reinterpret_cast<bf16(*)[BN + 8]>(sm + A_BYTES);
    const int split = blockIdx.z % splits, ph = blockIdx.z / splits;
    la.set_phase(ph);
    lb.set_phase(ph);
    ep.set_phase(ph);
    if constexpr (std::is_same<EP, EpPartial>::value) ep.split = split;
    const long long m0 = (long long)blockIdx.x * BM;
    const int n0 = blockIdx.y * BN;
    const int kbeg = split * k_split, kend = min(K, kbeg + k_split);
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int wm = warp & 3, wn = warp >> 2, g = lane >> 2, t = lane & 3;
    float acc[2][4][4];
#pragma unroll
    for (int i = 0; i < 2; ++i)
#pragma unroll
        for (int j = 0; j < 4; ++j)
#pragma unroll
            for (int q = 0; q < 4; ++q) acc[i][j][q] = 0.0f;
    la.prepare(m0, M);
    lb.prepare(n0, N);
    if (kbeg < kend) {
        la.fetch(kbeg, kend);
        lb.fetch(kbeg, kend);
    }
    for (int k0 = kbeg; k0 < kend; k0 += BK) {
        if constexpr (LA::KMAJOR) la.put(AsT);
        else la.put(As);
        if constexpr (LB::KMAJOR) lb.put(BsT);
        else lb.put(Bs);
        __syncthreads();
        if (k0 + BK < kend) {  // the next tile's loads, in flight during these MMAs
            la.fetch(k0 + BK, kend);
            lb.fetch(k0 + BK, kend);
        }
#pragma unroll
        for (int kk = 0; kk < BK; kk += 16) {
            uint32_t a[2][4], b[4][2];
            const int q = lane >> 3, rr = lane & 7;  // ldmatrix: matrix q, row rr
#pragma unroll
            for (int i = 0; i < 2; ++i) {
                const int r = wm * 32 + i * 16 + g;
                if constexpr (LA::KMAJOR) {
                    // matrices (k 0-7, m 0-7), (k 0-7, m 8-15), (k 8-15, m 0-7), (k 8-15, m 8-15)
                    ldmatrix_x4_trans(a[i], &AsT[kk + (q & 2) * 4 + rr][wm * 32 + i * 16 + (q & 1) * 8]);
                } else {
                    // matrices (m 0-7, k 0-7), (m 8-15, k 0-7), (m 0-7, k 8-15), (m 8-15, k 8-15)
                    (void)r;
                    ldmatrix_x4(a[i], &As[wm * 32 + i * 16 + (q & 1) * 8 + rr][kk + (q & 2) * 4]);
                }
            }
#pragma unroll
            for (int j = 0; j < 4; ++j) {
                if constexpr (LB::KMAJOR) {
                    if (j % 2 == 0) {
                        // matrices (k 0-7, n 0-7), (k 8-15, n 0-7), (k 0-7, n 8-15), (k 8-15, n 8-15)
                        uint32_t r4[4];
                        ldmatrix_x4_trans(r4, &BsT[kk + (q & 1) * 8 + rr][wn * 32 + j * 8 + (q & 2) * 4]);
                        b[j][0] = r4[0];
                        b[j][1] = r4[1];
                        b[j + 1][0] = r4[2];
                        b[j + 1][1] = r4[3];
                    }
                } else if (j % 2 == 0) {
                    // matrices (n 0-7, k 0-7), (n 0-7, k 8-15), (n 8-15, k 0-7), (n 8-15, k 8-15)
                    uint32_t r4[4];
                    ldmatrix_x4(r4, &Bs[wn * 32 + j * 8 + (q & 2) * 4 + rr][kk + (q & 1) * 8]);
                    b[j][0] = r4[0];
                    b[j][1] = r4[1];
                    b[j + 1][0] = r4[2];
                    b[j + 1][1] = r4[3];
                }
            }
#pragma unroll
            for (int i = 0; i < 2; ++i)
#pragma unroll
                for (int j = 0; j < 4; ++j) mma16816(acc[i][j], a[i], b[j]);
        }
        __syncthreads();
    }
#pragma unroll
    for (int i = 0; i < 2; ++i)
#pragma unroll
        for (int j = 0; j < 4; ++j) {
            const long long r0 = m0 + wm * 32 + i * 16 + g;
            const int c = n0 + wn * 32 + j * 8 + 2 * t;
            if (c >= N) continue;
            if (r0 < M) ep.store(r0, c, acc[i][j][0], acc[i][j][1]);
            if (r0 + 8 < M) ep.store(r0 + 8, c, acc[i][j][2], acc[i][j][3]);
        }
}

// ------------------------------------------------ tcgen05 convolution GEMM
//
// The convolution GEMMs whose A operand is an image gathered through taps
// (3x3 convolution and its input gradient, the 1-tap products of the
// transposed convolution) on the Blackwell tensor cores: a CTA computes a
// 128-pixel x BN-channel tile of C, the pixels a 16 x 8 patch of one image
// (width a multiple of 16, height of 8).  K runs over (tap, channel chunk of
// KC).  For each step one thread issues two TMA copies into a ring of
// shared-memory stages: the A box (KC channels, 16 x 8 pixels shifted by the
// tap) of a 4D map over the NHWC activations, whose out-of-image pixels and
// channels beyond C_in the copy engine fills with zeros (the convolution's
// zero padding), and the B box (KC columns, BN rows) of the prepared weights.
// A second thread issues the tcgen05.mma steps (128 x BN x 16 each) into an
// FP32 accumulator in tensor memory and releases each stage through
// tcgen05.commit on its mbarrier.  The four warps then read the accumulator
// back (tcgen05.ld, one pixel row per thread) through the same epilogues as
// k_gemm.  Every wait is bounded in time: a wait that gives up sets a bit in
// g_umma_status, the CTA stops issuing, waits (bounded) for what it issued,
// frees its tensor memory and returns; later launches return at entry until
// unet_get_status reads the flag.
struct UmmaShape {
    int H, W, C;       // A: image height, width and channels
    int taps;          // 9 (3x3, zero padding) or 1
    int kc_per_tap;    // channel chunks per tap
    int N;             // output columns
    int rows_per_phase;  // B rows per phase (the phase's weight block)
};

__device__ unsigned g_umma_status;
constexpr unsigned kUmmaTimeout = 1u;
constexpr uint64_t kUmmaWaitNs = 500000000ull;  // 0.5 s per wait (a copy or an MMA step takes microseconds)
constexpr int kUmmaStages = 4;

template <int KC, int BN>
struct UmmaSmem {
    static constexpr int A_BYTES = 128 * KC * 2, B_BYTES = BN * KC * 2, STAGE = A_BYTES + B_BYTES;
    static constexpr int BARS = 2 * kUmmaStages + 1;
    static constexpr int BYTES = 1024 + kUmmaStages * STAGE + BARS * 8 + 16;  // + alignment slack
    static_assert(A_BYTES % 1024 == 0 && B_BYTES % 1024 == 0, "stage tiles keep the swizzle atoms 1024-B aligned");
};

template <int KC, int BN, class EP>
__global__ void __launch_bounds__(128, 1) k_umma_conv(const __grid_constant__ CUtensorMap ta,
                                                      const __grid_constant__ CUtensorMap tb, EP ep, UmmaShape sh)
{
    using SM = UmmaSmem<KC, BN>;
    namespace U = umma;
    // a wait of an earlier launch gave up (flag not yet read by unet_get_status): do nothing, so that one
    // failure costs one wait limit, not one per CTA
    if (*reinterpret_cast<volatile unsigned*>(&g_umma_status)) return;
    extern __shared__ unsigned char dyn[];
    const uint32_t s0 = U::smem_addr(dyn);
    unsigned char* base = dyn + ((1024u - (s0 & 1023u)) & 1023u);  // 1024-B aligned: the 128-byte swizzle atoms
    uint64_t* full = reinterpret_cast<uint64_t*>(base + kUmmaStages * SM::STAGE);
    uint64_t* empty = full + kUmmaStages;
    uint64_t* done = empty + kUmmaStages;
    uint32_t* tslot = reinterpret_cast<uint32_t*>(done + 1);
    volatile int* abort = reinterpret_cast<volatile int*>(tslot + 1);
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    if (threadIdx.x == 0) {
        for (int st = 0; st < kUmmaStages; ++st) {
            U::bar_init(&full[st], 1);
            U::bar_init(&empty[st], 1);
        }
        U::bar_init(done, 1);
        *abort = 0;
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    if (warp == 0) U::tmem_alloc(tslot, BN);
    U::fence_before_sync();
    __syncthreads();
    U::fence_after_sync();
    const uint32_t tmem = *tslot;
    // the tile: pixels (b, y0 .. y0 + 7, x0 .. x0 + 15), columns n0 .. n0 + BN - 1 of phase ph
    const int tw = sh.W / 16, tpi = tw * (sh.H / 8);
    const int b = blockIdx.x / tpi, r = blockIdx.x % tpi;
    const int y0 = (r / tw) * 8, x0 = (r % tw) * 16;
    const int n0 = blockIdx.y * BN, ph = blockIdx.z;
    ep.set_phase(ph);
    const int nk = sh.taps * sh.kc_per_tap;
    if (warp == 0 && lane == 0) {  // producer: TMA copies into the stage ring
        int it = 0;
        for (; it < nk; ++it) {
            const int st = it % kUmmaStages;
            if (it >= kUmmaStages &&
                !U::bar_wait(&empty[st], (uint32_t)(it / kUmmaStages - 1) & 1u, abort, &g_umma_status,
                             kUmmaTimeout, kUmmaWaitNs))
                break;
            const int tap = it / sh.kc_per_tap, kc = it - tap * sh.kc_per_tap;
            const int dy = sh.taps == 9 ? tap / 3 - 1 : 0, dx = sh.taps == 9 ? tap % 3 - 1 : 0;
            unsigned char* sa = base + st * SM::STAGE;
            U::bar_expect_tx(&full[st], SM::STAGE);
            U::tma_4d(sa, &ta, &full[st], kc * KC, x0 + dx, y0 + dy, b);
            U::tma_2d(sa + SM::A_BYTES, &tb, &full[st], tap * sh.C + kc * KC, ph * sh.rows_per_phase + n0);
        }
        // no copy may still be writing into shared memory when the CTA exits
        for (int j = it > kUmmaStages ? it - kUmmaStages : 0; j < it; ++j) {
            const uint64_t t0 = U::now_ns();
            while (!U::bar_test(&full[j % kUmmaStages], (uint32_t)(j / kUmmaStages) & 1u))
                if (U::now_ns() - t0 > kUmmaWaitNs) break;
        }
    } else if (warp == 1 && lane == 0) {  // MMA issuer
        constexpr uint32_t idesc = U::idesc_bf16_m128(BN);
        for (int it = 0; it < nk; ++it) {
            const int st = it % kUmmaStages;
            if (!U::bar_wait(&full[st], (uint32_t)(it / kUmmaStages) & 1u, abort, &g_umma_status, kUmmaTimeout,
                             kUmmaWaitNs))
                break;
            U::fence_after_sync();
            const uint32_t sa = U::smem_addr(base + st * SM::STAGE), sb = sa + SM::A_BYTES;
#pragma unroll
            for (int kk = 0; kk < KC / 16; ++kk)  // 16 bf16 = 32 bytes along K within the swizzle atom
                U::mma_bf16(tmem, U::kmajor_desc<KC>(sa + 32 * kk), U::kmajor_desc<KC>(sb + 32 * kk), idesc,
                            (it > 0 || kk > 0) ? 1u : 0u);
            U::mma_commit(&empty[st]);  // the stage is free once these steps have read it
        }
        U::mma_commit(done);  // every step issued above has completed
    }
    // epilogue: thread t of warp w holds pixel row 32 w + t of the tile
    U::bar_wait(done, 0, abort, &g_umma_status, kUmmaTimeout, kUmmaWaitNs);
    __syncthreads();  // the issuing threads are past their loops: `done` is committed
    U::fence_after_sync();
    const bool ok = !*abort;
    if (!ok) {  // a wait gave up: let the steps issued so far finish (bounded) before the memory is freed
        if (threadIdx.x == 0) {
            const uint64_t t0 = U::now_ns();
            while (!U::bar_test(done, 0))
                if (U::now_ns() - t0 > kUmmaWaitNs) break;
        }
        __syncthreads();
    }
    if (ok) {
        const int row = warp * 32 + lane;
        const long long p = ((long long)b * sh.H + y0 + row / 16) * sh.W + x0 + row % 16;
        __syncwarp();
#pragma unroll 1
        for (int c = 0; c < BN; c += 32) {
            uint32_t v[32];
            U::tmem_load32(tmem + ((uint32_t)(warp * 32) << 16) + (uint32_t)c, v);
#pragma unroll
            for (int j = 0; j < 32; j += 8) {  // N is a multiple of 32: eight columns are all in range or none
                const int n = n0 + c + j;
                if (n >= sh.N) continue;
                float f[8];
#pragma unroll
                for (int q = 0; q < 8; ++q) f[q] = __uint_as_float(v[j + q]);
                ep.store8(p, n, f);
            }
        }
    }
    U::fence_before_sync();
    __syncthreads();
    if (warp == 0) {
        __syncwarp();
        U::tmem_free(tmem, BN);
    }
}

// Weight gradient of a 3x3 convolution on the tensor cores:
// dW[(tap, ci)][co] = sum_p X[p + tap][ci] G[p][co], M = 9 C_in rows, N = C_out,
// K = the pixels.  K advances in chunks of 64 pixels (a 16 x 4 patch of one
// image); a CTA sums a contiguous range of chunks (its split) for a 128-row x
// BN-column tile and writes FP32 partials (EpPartial) that k_sum_partials adds
// in a fixed order.  Both operands are MN-major: a TMA box of AW channels x
// 16 x 4 pixels of the NHWC tensor lands as 64 rows (pixels, the K index) of
// AW channels (AW = 64: 128-byte rows, 128-byte swizzle; AW = 32: 64-byte
// rows, 64-byte swizzle), eight rows per atom; the A tile is 128 / AW such
// boxes (AW rows (tap, ci) each, one tap per box: C_in is a multiple of AW),
// the B tile BN / BW boxes of G.  Pipeline, waits and epilogue as in
// k_umma_conv.  With up = 1 the same kernel gives the weight gradient of the
// 2x2 stride-2 transposed convolution, dW[phase][ci][co] = sum_p X[p][ci]
// G[up(p, phase)][co]: one tap, the phase from blockIdx.z / splits, and G's
// box holds that phase's samples of the output gradient, read through a 5D
// map (channel, x parity, x pair, y parity, image row pair) so that a plain
// box selects them.
struct UmmaWgrad {
    int H, W, Cin, N;
    long long M;                // 9 C_in (3x3), C_in (transposed convolution)
    int chunks_per_image;       // (H / 4) (W / 16)
    long long chunks;           // over the batch
    int chunks_per_split;
    int up;                     // 1: transposed convolution, one product per output phase (blockIdx.z / splits)
    int splits;
};

template <int AW, int BN, int BW>
struct WgradSmem {
    static constexpr int ABOX = 64 * AW * 2, BBOX = 64 * BW * 2;  // 64 pixels x the block's channels
    static constexpr int ABLK = 128 / AW, BBLK = BN / BW;
    static constexpr int A_BYTES = ABLK * ABOX, B_BYTES = BBLK * BBOX, STAGE = A_BYTES + B_BYTES;
    static constexpr int BYTES = 1024 + kUmmaStages * STAGE + (2 * kUmmaStages + 1) * 8 + 16;
    static_assert(STAGE % 1024 == 0, "stage tiles keep the swizzle atoms aligned");
};

template <int AW, int BN, int BW>
__global__ void __launch_bounds__(128, 1) k_umma_wgrad(const __grid_constant__ CUtensorMap tx,
                                                       const __grid_constant__ CUtensorMap tg, EpPartial ep,
                                                       UmmaWgrad sh)
{
    using WS = WgradSmem<AW, BN, BW>;
    constexpr int A_BYTES = WS::A_BYTES, STAGE = WS::STAGE;
    namespace U = umma;
    if (*reinterpret_cast<volatile unsigned*>(&g_umma_status)) return;
    extern __shared__ unsigned char dyn[];
    const uint32_t s0 = U::smem_addr(dyn);
    unsigned char* base = dyn + ((1024u - (s0 & 1023u)) & 1023u);
    uint64_t* full = reinterpret_cast<uint64_t*>(base + kUmmaStages * STAGE);
    uint64_t* empty = full + kUmmaStages;
    uint64_t* done = empty + kUmmaStages;
    uint32_t* tslot = reinterpret_cast<uint32_t*>(done + 1);
    volatile int* abort = reinterpret_cast<volatile int*>(tslot + 1);
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    if (threadIdx.x == 0) {
        for (int st = 0; st < kUmmaStages; ++st) {
            U::bar_init(&full[st], 1);
            U::bar_init(&empty[st], 1);
        }
        U::bar_init(done, 1);
        *abort = 0;
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    if (warp == 0) U::tmem_alloc(tslot, BN);
    U::fence_before_sync();
    __syncthreads();
    U::fence_after_sync();
    const uint32_t tmem = *tslot;
    const long long m0 = (long long)blockIdx.x * 128;
    const int n0 = blockIdx.y * BN;
    const int split = sh.up ? (int)(blockIdx.z % sh.splits) : (int)blockIdx.z;
    const int ph = sh.up ? (int)(blockIdx.z / sh.splits) : 0;
    ep.split = split;
    ep.set_phase(ph);
    const long long c0 = (long long)split * sh.chunks_per_split;
    const int nk = (int)max(0LL, min(sh.chunks, c0 + sh.chunks_per_split) - c0);
    // the A tile's AW-row blocks: tap and first channel of each, and whether it holds any row
    int tap[WS::ABLK], ci[WS::ABLK];
    bool live[WS::ABLK];
    uint32_t bytes = WS::B_BYTES;
#pragma unroll
    for (int j = 0; j < WS::ABLK; ++j) {
        const long long r0 = m0 + AW * j;
        live[j] = r0 < sh.M;
        tap[j] = live[j] && !sh.up ? (int)(r0 / sh.Cin) : 4;  // tap 4: no shift
        ci[j] = live[j] ? (int)(r0 % sh.Cin) : 0;
        bytes += live[j] ? WS::ABOX : 0;
    }
    const int tw = sh.W / 16;
    if (warp == 0 && lane == 0) {  // producer
        int it = 0;
        for (; it < nk; ++it) {
            const int st = it % kUmmaStages;
            if (it >= kUmmaStages &&
                !U::bar_wait(&empty[st], (uint32_t)(it / kUmmaStages - 1) & 1u, abort, &g_umma_status,
                             kUmmaTimeout, kUmmaWaitNs))
                break;
            const long long c = c0 + it;
            const int b = (int)(c / sh.chunks_per_image), r = (int)(c % sh.chunks_per_image);
            const int y0 = (r / tw) * 4, x0 = (r % tw) * 16;
            unsigned char* sa = base + st * STAGE;
            U::bar_expect_tx(&full[st], bytes);
#pragma unroll
            for (int j = 0; j < WS::ABLK; ++j)
                if (live[j])
                    U::tma_4d(sa + j * WS::ABOX, &tx, &full[st], ci[j], x0 + tap[j] % 3 - 1, y0 + tap[j] / 3 - 1, b);
#pragma unroll
            for (int j = 0; j < WS::BBLK; ++j) {
                if (sh.up)
                    U::tma_5d(sa + A_BYTES + j * WS::BBOX, &tg, &full[st], n0 + BW * j, ph & 1, x0, ph >> 1,
                              b * sh.H + y0);
                else
                    U::tma_4d(sa + A_BYTES + j * WS::BBOX, &tg, &full[st], n0 + BW * j, x0, y0, b);
            }
        }
        for (int j = it > kUmmaStages ? it - kUmmaStages : 0; j < it; ++j) {
            const uint64_t t0 = U::now_ns();
            while (!U::bar_test(&full[j % kUmmaStages], (uint32_t)(j / kUmmaStages) & 1u))
                if (U::now_ns() - t0 > kUmmaWaitNs) break;
        }
    } else if (warp == 1 && lane == 0) {  // MMA issuer
        constexpr uint32_t idesc = U::idesc_bf16_m128(BN, true, true);
        for (int it = 0; it < nk; ++it) {
            const int st = it % kUmmaStages;
            if (!U::bar_wait(&full[st], (uint32_t)(it / kUmmaStages) & 1u, abort, &g_umma_status, kUmmaTimeout,
                             kUmmaWaitNs))
                break;
            U::fence_after_sync();
            const uint32_t sa = U::smem_addr(base + st * STAGE), sb = sa + A_BYTES;
#pragma unroll
            for (int kk = 0; kk < 4; ++kk)  // 16 pixels (two 8-row groups) per step
                U::mma_bf16(tmem, U::mnmajor_desc<AW>(sa + 16 * AW * 2 * kk, WS::ABOX),
                            U::mnmajor_desc<BW>(sb + 16 * BW * 2 * kk, WS::BBOX), idesc, (it > 0 || kk > 0) ? 1u : 0u);
            U::mma_commit(&empty[st]);
        }
        U::mma_commit(done);
    }
    U::bar_wait(done, 0, abort, &g_umma_status, kUmmaTimeout, kUmmaWaitNs);
    __syncthreads();
    U::fence_after_sync();
    const bool ok = !*abort;
    if (!ok) {
        if (threadIdx.x == 0) {
            const uint64_t t0 = U::now_ns();
            while (!U::bar_test(done, 0))
                if (U::now_ns() - t0 > kUmmaWaitNs) break;
        }
        __syncthreads();
    }
    if (ok) {
        const long long m = m0 + warp * 32 + lane;
        __syncwarp();
#pragma unroll 1
        for (int c = 0; c < BN; c += 32) {
            uint32_t v[32];
            if (nk > 0) {
                U::tmem_load32(tmem + ((uint32_t)(warp * 32) << 16) + (uint32_t)c, v);
            } else {  // an empty split: its partial is zero
#pragma unroll
                for (int j = 0; j < 32; ++j) v[j] = 0u;
            }
            if (m < sh.M) {
#pragma unroll
                for (int j = 0; j < 32; j += 8) {  // N is a multiple of 32
                    const int n = n0 + c + j;
                    if (n >= sh.N) continue;
                    float f[8];
#pragma unroll
                    for (int q = 0; q < 8; ++q) f[q] = __uint_as_float(v[j + q]);
                    ep.store8(m, n, f);
                }
            }
        }
    }
    U::fence_before_sync();
    __syncthreads();
    if (warp == 0) {
        __syncwarp();
        U::tmem_free(tmem, BN);
    }
}

// ------------------------------------------------------ elementwise kernels

__global__ void k_sum_partials(const float* __restrict__ part, long long count, int splits, long long stride,
                               float* __restrict__ out)
{
    for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < count; i += (long long)gridDim.x * blockDim.x) {
        float s = 0.0f;
        for (int k = 0; k < splits; ++k) s += part[k * stride + i];
        out[i] = s;
    }
}

// The same for few outputs over many splits: one warp per output, lane l
// adding splits l, l + 32, ... in order, then a fixed butterfly.
__global__ void __launch_bounds__(256) k_sum_partials_warp(const float* __restrict__ part, long long count,
                                                           int splits, long long stride, float* __restrict__ out)
{
    const long long i = (long long)blockIdx.x * 8 + (threadIdx.x >> 5);
    const int lane = threadIdx.x & 31;
    if (i >= count) return;
    float s = 0.0f;
    for (int k = lane; k < splits; k += 32) s += part[k * stride + i];
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
    if (lane == 0) out[i] = s;
}

unsigned ew_grid(long long n);

void sum_partials(cudaStream_t st, const float* part, long long count, int splits, long long stride, float* out)
{
    if (count <= 16384 && splits >= 16)
        k_sum_partials_warp<<<(unsigned)((count + 7) / 8), 256, 0, st>>>(part, count, splits, stride, out);
    else
        k_sum_partials<<<ew_grid(count), 256, 0, st>>>(part, count, splits, stride, out);
}

// Eight bf16 (16 bytes) at a time: C, row strides and channel offsets are
// multiples of 8 throughout the network.
union V8 {
    uint4 u;
    bf16 h[8];
};

__device__ __forceinline__ V8 ld8(const bf16* p)
{
    V8 v;
    v.u = *reinterpret_cast<const uint4*>(p);
    return v;
}

__device__ __forceinline__ void st8(bf16* p, const V8& v) { *reinterpret_cast<uint4*>(p) = v.u; }

// Column sums of g[P][C] (row stride ld, channel offset off) over a range of
// rows per block: part[block][c].  Thread (group rg, vector cv) adds the rows
// rg, rg + RG, ... of channels 8 cv .. 8 cv + 7 (RG = 256 / (C / 8) groups);
// the groups are then added in order through shared memory.  C / 8 divides
// 256 (C = 8 2^k, C <= 2048).
__global__ void __launch_bounds__(256) k_colsum(const bf16* __restrict__ g, long long P, int C, int ld, int off,
                                                long long rows, float* __restrict__ part)
{
    __shared__ float red[256 * 8];
    const int nv = C / 8, RG = 256 / nv, rg = threadIdx.x / nv, cv = threadIdx.x % nv;
    const long long r0 = (long long)blockIdx.x * rows, r1 = min(P, r0 + rows);
    float acc[8] = {0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f};
    for (long long r = r0 + rg; r < r1; r += RG) {
        const V8 v = ld8(g + r * ld + off + 8 * cv);
#pragma unroll
        for (int j = 0; j < 8; ++j) acc[j] += __bfloat162float(v.h[j]);
    }
#pragma unroll
    for (int j = 0; j < 8; ++j) red[threadIdx.x * 8 + j] = acc[j];
    __syncthreads();
    for (int c = threadIdx.x; c < C; c += 256) {
        float t = 0.0f;
        for (int q = 0; q < RG; ++q) t += red[(q * nv + c / 8) * 8 + c % 8];
        part[(long long)blockIdx.x * C + c] = t;
    }
}

// out[p][c] = dy[p][off + c] * (y[p][c] > 0)
__global__ void k_relu_grad(const bf16* __restrict__ dy, int ld_dy, int off_dy, const bf16* __restrict__ y,
                            bf16* __restrict__ out, long long P, int C)
{
    const int nv = C / 8;
    const long long n = P * nv;
    for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x) {
        const long long p = i / nv;
        const int c = (int)(i - p * nv) * 8;
        const V8 d = ld8(dy + p * ld_dy + off_dy + c), a = ld8(y + p * C + c);
        V8 o;
#pragma unroll
        for (int j = 0; j < 8; ++j) o.h[j] = __bfloat162float(a.h[j]) > 0.0f ? d.h[j] : __float2bfloat16(0.0f);
        st8(out + p * C + c, o);
    }
}

// 2x2 max-pool of x[B][H][W][C] (first maximum in tap order), tap index kept.
__global__ void k_maxpool(const bf16* __restrict__ x, int B, int H, int W, int C, bf16* __restrict__ y,
                          uint8_t* __restrict__ arg)
{
    const int Ho = H / 2, Wo = W / 2, nv = C / 8;
    const long long n = (long long)B * Ho * Wo * nv;
    for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x) {
        const long long q = i / nv;
        const int c = (int)(i - q * nv) * 8;
        const int xo = (int)(q % Wo), yo = (int)((q / Wo) % Ho);
        const long long b = q / ((long long)Wo * Ho);
        float best[8];
        uint8_t bt[8];
#pragma unroll
        for (int t = 0; t < 4; ++t) {
            const V8 v = ld8(x + (((b * H) + 2 * yo + t / 2) * W + 2 * xo + t % 2) * C + c);
#pragma unroll
            for (int j = 0; j < 8; ++j) {
                const float f = __bfloat162float(v.h[j]);
                if (t == 0 || f > best[j]) {
                    best[j] = f;
                    bt[j] = (uint8_t)t;
                }
            }
        }
        V8 o;
        uint2 ar;
        uint8_t* a8 = reinterpret_cast<uint8_t*>(&ar);
#pragma unroll
        for (int j = 0; j < 8; ++j) {
            o.h[j] = __float2bfloat16(best[j]);
            a8[j] = bt[j];
        }
        st8(y + q * C + c, o);
        *reinterpret_cast<uint2*>(arg + q * C + c) = ar;
    }
}

// dx[B][H][W][C] = scatter of dy at the max-pool taps + skip[...][off + c] (row stride ld_s)
__global__ void k_maxpool_grad(const bf16* __restrict__ dy, const uint8_t* __restrict__ arg, int B, int H, int W,
                               int C, const bf16* __restrict__ skip, int ld_s, int off_s, bf16* __restrict__ dx)
{
    const int Ho = H / 2, Wo = W / 2, nv = C / 8;
    const long long n = (long long)B * H * W * nv;
    for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x) {
        const long long p = i / nv;
        const int c = (int)(i - p * nv) * 8;
        const int xx = (int)(p % W), yy = (int)((p / W) % H);
        const long long b = p / ((long long)W * H);
        const long long o = (((b * Ho) + yy / 2) * Wo + xx / 2) * C + c;
        const int t = (yy % 2) * 2 + (xx % 2);
        const V8 d = ld8(dy + o), sk = ld8(skip + p * ld_s + off_s + c);
        const uint2 ar = *reinterpret_cast<const uint2*>(arg + o);
        const uint8_t* a8 = reinterpret_cast<const uint8_t*>(&ar);
        V8 r;
#pragma unroll
        for (int j = 0; j < 8; ++j) {
            const float v = (a8[j] == t ? __bfloat162float(d.h[j]) : 0.0f) + __bfloat162float(sk.h[j]);
            r.h[j] = __float2bfloat16(v);
        }
        st8(dx + p * C + c, r);
    }
}

// dst[p][off + c] = src[p][c]
__global__ void k_copy_channels(const bf16* __restrict__ src, long long P, int C, bf16* __restrict__ dst, int ld,
                                int off)
{
    const int nv = C / 8;
    const long long n = P * nv;
    for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x) {
        const long long p = i / nv;
        const int c = (int)(i - p * nv) * 8;
        st8(dst + p * ld + off + c, ld8(src + p * C + c));
    }
}

// out[b][h] = mean_w (sum_c x[b][h][w][c] w[c] + bias): one block per row (b, h).
__global__ void k_head(const bf16* __restrict__ x, int W, int C, const float* __restrict__ w,
                       const float* __restrict__ bias, float* __restrict__ out)
{
    const long long row = blockIdx.x;
    float s = 0.0f;
    for (int i = threadIdx.x; i < W * C; i += blockDim.x) s += __bfloat162float(x[row * W * C + i]) * w[i % C];
    __shared__ float red[32];
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
    if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = s;
    __syncthreads();
    if (threadIdx.x == 0) {
        float t = 0.0f;
        for (int i = 0; i < (int)(blockDim.x >> 5); ++i) t += red[i];
        out[row] = t / (float)W + bias[0];
    }
}

// Loss mean((out - target)^2) and gout = 2 (out - target) / n (one block).
__global__ void k_mse(const float* __restrict__ out, const float* __restrict__ target, int n, float* __restrict__ loss,
                      float* __restrict__ gout)
{
    float s = 0.0f;
    for (int i = threadIdx.x; i < n; i += blockDim.x) {
        const float d = out[i] - target[i];
        s += d * d;
        gout[i] = 2.0f * d / (float)n;
    }
    __shared__ float red[32];
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
    if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = s;
    __syncthreads();
    if (threadIdx.x == 0) {
        float t = 0.0f;
        for (int i = 0; i < (int)(blockDim.x >> 5); ++i) t += red[i];
        *loss = t / (float)n;
    }
}

// Head backward, one block per row (b, h): dx[b][h][w][c] = gout[b][h] / W * w[c];
// part_w[row][c] = sum_w x[b][h][w][c] gout / W.
__global__ void __launch_bounds__(256) k_head_grad(const bf16* __restrict__ x, int W, int C,
                                                   const float* __restrict__ w, const float* __restrict__ gout,
                                                   bf16* __restrict__ dx, float* __restrict__ part_w)
{
    __shared__ float red[256];
    const long long row = blockIdx.x;
    const float gr = gout[row] / (float)W;
    const int nv = C / 8;
    for (int i = threadIdx.x; i < W * nv; i += blockDim.x) {
        const int c = (i % nv) * 8;
        V8 o;
#pragma unroll
        for (int j = 0; j < 8; ++j) o.h[j] = __float2bfloat16(gr * w[c + j]);
        st8(dx + row * W * C + (long long)i * 8, o);
    }
    // part_w[row][c] = gr * sum_w x[row][w][c]: thread (group xg, channel c) adds w = xg, xg + XG, ...; the groups
    // are added in order (C <= 256)
    const int XG = 256 / C, xg = threadIdx.x / C, c = threadIdx.x % C;
    float s = 0.0f;
    if (xg < XG)
        for (int xw = xg; xw < W; xw += XG) s += __bfloat162float(x[(row * W + xw) * C + c]);
    red[threadIdx.x] = s;
    __syncthreads();
    if (threadIdx.x < C) {
        float t = 0.0f;
        for (int q = 0; q < XG; ++q) t += red[q * C + threadIdx.x];
        part_w[row * C + threadIdx.x] = t * gr;
    }
}

// *out = sum of v[0 .. n) (one block of 256 threads, fixed order).
__global__ void __launch_bounds__(256) k_sum_vector(const float* __restrict__ v, int n, float* __restrict__ out)
{
    __shared__ float red[256];
    float s = 0.0f;
    for (int i = threadIdx.x; i < n; i += 256) s += v[i];
    red[threadIdx.x] = s;
    __syncthreads();
    for (int o = 128; o > 0; o >>= 1) {
        if ((int)threadIdx.x < o) red[threadIdx.x] += red[threadIdx.x + o];
        __syncthreads();
    }
    if (threadIdx.x == 0) *out = red[0];
}

// Input packing: x[b][h][w][c] = (u_x s, u_y s, mask, 0 ...).
__global__ void k_pack(const double* __restrict__ u, const uint8_t* __restrict__ mask, int B, int H, int W,
                       float scale, bf16* __restrict__ x)
{
    const long long n = (long long)B * H * W;
    for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x) {
        const long long b = i / ((long long)H * W), hw = i - b * H * W;
        bf16* o = x + i * UNET_IN_CHANNELS;
        o[0] = __float2bfloat16((float)u[(b * 2 + 0) * H * W + hw] * scale);
        o[1] = __float2bfloat16((float)u[(b * 2 + 1) * H * W + hw] * scale);
        o[2] = __float2bfloat16(mask[i] ? 1.0f : 0.0f);
#pragma unroll
        for (int c = 3; c < UNET_IN_CHANNELS; ++c) o[c] = __float2bfloat16(0.0f);
    }
}

// FP32 master [taps][Cin][Cout] -> fwd[co][tap * Cin + ci] and
// bwd[ci][tap' * Cout + co] (tap' = taps - 1 - tap for a 3x3 kernel: the
// input gradient is the correlation with the flipped kernel; for the
// transposed convolution tap' = tap, fwd is [phase][co][ci]).
__global__ void k_prep_weights(const float* __restrict__ w, int taps, int Cin, int Cout, int flip, int phase_major,
                               bf16* __restrict__ fwd, bf16* __restrict__ bwd)
{
    const long long n = (long long)taps * Cin * Cout;
    for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x) {
        const int co = (int)(i % Cout), ci = (int)((i / Cout) % Cin), tap = (int)(i / ((long long)Cout * Cin));
        const bf16 v = __float2bfloat16(w[i]);
        if (phase_major) fwd[((long long)tap * Cout + co) * Cin + ci] = v;
        else fwd[(long long)co * taps * Cin + (long long)tap * Cin + ci] = v;
        const int tb = flip ? taps - 1 - tap : tap;
        bwd[(long long)ci * taps * Cout + (long long)tb * Cout + co] = v;
    }
}

__global__ void k_adam_f32(long long n, float* __restrict__ p, float* __restrict__ m, float* __restrict__ v,
                           const float* __restrict__ g, float lr, float b1, float b2, float eps, float c1, float c2)
{
    for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x) {
        const float gi = g[i];
        const float mi = b1 * m[i] + (1.0f - b1) * gi;
        const float vi = b2 * v[i] + (1.0f - b2) * gi * gi;
        m[i] = mi;
        v[i] = vi;
        p[i] -= lr * (mi / c1) / (sqrtf(vi / c2) + eps);
    }
}

// ------------------------------------------------------------ host side

unsigned ew_grid(long long n) { return (unsigned)std::max<long long>(1, std::min<long long>((n + 255) / 256, 152 * 16)); }

struct Tensor {
    int64_t off, count;
};

// Parameter tensors in the order of unet.h.
std::vector<Tensor> param_tensors(int base, std::vector<int>* taps_out = nullptr, std::vector<int>* cin_out = nullptr,
                                  std::vector<int>* cout_out = nullptr)
{
    std::vector<Tensor> t;
    std::vector<int> taps, cin, cout;
    int64_t o = 0;
    auto add = [&](int tp, int ci, int co) {
        t.push_back({o, (int64_t)tp * ci * co});
        o += (int64_t)tp * ci * co;
        taps.push_back(tp), cin.push_back(ci), cout.push_back(co);
        t.push_back({o, co});  // bias
        o += co;
        taps.push_back(0), cin.push_back(0), cout.push_back(co);
    };
    const int c[4] = {base, 2 * base, 4 * base, 8 * base};
    int prev = UNET_IN_CHANNELS;
    for (int l = 0; l < 4; ++l) {
        add(9, prev, c[l]);
        add(9, c[l], c[l]);
        prev = c[l];
    }
    for (int l = 2; l >= 0; --l) {
        add(4, c[l + 1], c[l]);
        add(9, 2 * c[l], c[l]);
        add(9, c[l], c[l]);
    }
    t.push_back({o, base});
    o += base;
    taps.push_back(1), cin.push_back(base), cout.push_back(1);
    t.push_back({o, 1});
    taps.push_back(0), cin.push_back(0), cout.push_back(1);
    if (taps_out) *taps_out = taps;
    if (cin_out) *cin_out = cin;
    if (cout_out) *cout_out = cout;
    return t;
}

constexpr int kMaxSplits = 256;
constexpr long long kTargetCtas = 608;  // weight-gradient CTAs aimed for (4 per SM)

struct Layout {
    int B, H, W, c[4];
    int Hl[4], Wl[4];
    long long P[4];                              // pixels per level (all samples)
    size_t wf[17], wb[17];                       // bf16 operand layouts of the 17 convolution layers (forward order)
    size_t bias;                                 // FP32 copy of all parameters (biases and head read from it)
    size_t ea[4], eb[4], pool[3], arg[3], cat[3], da[3], db[3];
    size_t out, gout, loss_tmp;
    size_t gA, gB, gC, gcat[3];
    size_t part;                                 // split-K / column-sum partials (FP32)
    long long part_floats;
    size_t total;
    int64_t n_params;
};

size_t al256(size_t x) { return (x + 255) & ~size_t(255); }

bool make_layout(const unet_desc* d, Layout* L)
{
    if (!d || d->base < 8 || d->base % 8 || d->height < 8 || d->height % 8 || d->width < 8 || d->width % 8 ||
        d->batch < 1 || d->base > 256)
        return false;
    Layout& l = *L;
    l.B = d->batch;
    l.H = d->height;
    l.W = d->width;
    for (int i = 0; i < 4; ++i) {
        l.c[i] = d->base << i;
        l.Hl[i] = l.H >> i;
        l.Wl[i] = l.W >> i;
        l.P[i] = (long long)l.B * l.Hl[i] * l.Wl[i];
    }
    std::vector<int> taps, cin, cout;
    const auto t = param_tensors(d->base, &taps, &cin, &cout);
    l.n_params = t.back().off + t.back().count;
    size_t o = 0;
    int wi = 0;
    long long max_part = 0;
    for (size_t i = 0; i + 2 < t.size(); i += 2) {  // weight tensors of the 11 layers
        const size_t bytes = al256(sizeof(bf16) * (size_t)t[i].count);
        l.wf[wi] = o;
        o += bytes;
        l.wb[wi] = o;
        o += bytes;
        ++wi;
    }
    l.bias = o;
    o += al256(sizeof(float) * (size_t)l.n_params);
    auto act = [&](long long P, int C) {
        const size_t off = o;
        o += al256(sizeof(bf16) * (size_t)P * C);
        return off;
    };
    for (int i = 0; i < 4; ++i) {
        l.ea[i] = act(l.P[i], l.c[i]);
        l.eb[i] = act(l.P[i], l.c[i]);
    }
    for (int i = 0; i < 3; ++i) {
        l.pool[i] = act(l.P[i + 1], l.c[i]);
        l.arg[i] = o;
        o += al256((size_t)l.P[i + 1] * l.c[i]);
        l.cat[i] = act(l.P[i], 2 * l.c[i]);
        l.da[i] = act(l.P[i], l.c[i]);
        l.db[i] = act(l.P[i], l.c[i]);
        l.gcat[i] = act(l.P[i], 2 * l.c[i]);
    }
    long long gmax = 0;
    for (int i = 0; i < 4; ++i) gmax = std::max(gmax, l.P[i] * 2 * l.c[i]);
    l.gA = act(gmax, 1);
    l.gB = act(gmax, 1);
    l.gC = act(gmax, 1);
    l.out = o;
    o += al256(sizeof(float) * (size_t)l.B * l.H);
    l.gout = o;
    o += al256(sizeof(float) * (size_t)l.B * l.H);
    l.loss_tmp = o;
    o += 256;
    // partials: weight gradients (splits x (phases) x M x N: at most (kTargetCtas + tiles) x BM x BN, or the
    // largest product at 16 k-tiles per split), column sums (blocks x C), head (rows x c0)
    max_part = (kTargetCtas + 1) * BM * BN * 2;
    for (int i = 0; i < 4; ++i) {
        const long long cmax = 2LL * l.c[std::min(i + 1, 3)];
        max_part = std::max(max_part, 4 * 9 * cmax * cmax);
        max_part = std::max(max_part, 256LL * cmax);
    }
    max_part = std::max(max_part, (long long)l.B * l.H * l.c[0]);
    l.part = o;
    l.part_floats = max_part;
    o += al256(sizeof(float) * (size_t)max_part);
    l.total = o;
    return true;
}

template <class T>
T* at(void* ws, size_t off)
{
    return reinterpret_cast<T*>(static_cast<unsigned char*>(ws) + off);
}

struct Ctx {
    const Layout& L;
    void* ws;
    cudaStream_t s;
    std::vector<Tensor> t;
    bf16* wf(int layer) const { return at<bf16>(ws, L.wf[layer]); }
    bf16* wb(int layer) const { return at<bf16>(ws, L.wb[layer]); }
    const float* pw(int tensor) const { return at<float>(ws, L.bias) + t[tensor].off; }  // FP32 copy of a tensor
};

template <class LA, class LB, class EP>
void gemm(cudaStream_t s, const LA& la, const LB& lb, const EP& ep, long long M, int N, int K, int splits, int phases)
{
    const int k_split = ((K + splits - 1) / splits + BK - 1) / BK * BK;
    const dim3 grid((unsigned)((M + BM - 1) / BM), (unsigned)((N + BN - 1) / BN), (unsigned)(splits * phases));
    k_gemm<LA, LB, EP><<<grid, kGemmThreads, 0, s>>>(la, lb, ep, M, N, K, k_split, splits);
}

int g_engine = UNET_ENGINE_TCGEN05;

template <int KC, int BN, class EP>
bool launch_umma(cudaStream_t s, const CUtensorMap& ta, const CUtensorMap& tb, const EP& ep, const UmmaShape& sh,
                 dim3 grid)
{
    using SM = UmmaSmem<KC, BN>;
    static const bool attr = cudaFuncSetAttribute(k_umma_conv<KC, BN, EP>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                                  SM::BYTES) == cudaSuccess;
    if (!attr) return false;
    k_umma_conv<KC, BN, EP><<<grid, 128, SM::BYTES, s>>>(ta, tb, ep, sh);
    return cudaGetLastError() == cudaSuccess;
}

template <int KC, class EP>
bool launch_umma_bn(int bn, cudaStream_t s, const CUtensorMap& ta, const CUtensorMap& tb, const EP& ep,
                    const UmmaShape& sh, dim3 grid)
{
    switch (bn) {
    case 32: return launch_umma<KC, 32>(s, ta, tb, ep, sh, grid);
    case 64: return launch_umma<KC, 64>(s, ta, tb, ep, sh, grid);
    case 128: return launch_umma<KC, 128>(s, ta, tb, ep, sh, grid);
    default: return launch_umma<KC, 256>(s, ta, tb, ep, sh, grid);
    }
}

// The convolution product on the tensor cores (k_umma_conv), if the shapes
// allow it: A is the batch of Bimg images x (H x W pixels, C channels at row
// stride ld from channel off), gathered through `taps` taps; B the weights w
// ([phases][rows_per_phase][taps C], K contiguous); N output columns per
// phase.  false: the caller runs k_gemm instead (nothing was launched).
template <class EP>
bool umma_conv(cudaStream_t s, const bf16* x, int Bimg, int H, int W, int C, int ld, int off, int taps,
               const bf16* w, int rows_per_phase, int phases, int N, const EP& ep)
{
    if (g_engine != UNET_ENGINE_TCGEN05) return false;
    if (W % 16 || H % 8 || (C % 64 && C != 32) || N % 32 || ld % 8 || off % 8 || (taps != 9 && taps != 1))
        return false;
    umma::EncodeTiledFn enc = umma::tensor_map_encoder();
    if (!enc) return false;
    const int KC = C % 64 == 0 ? 64 : 32;
    const long long tiles_m = (long long)Bimg * (H / 8) * (W / 16);
    // widest tile that N allows, narrowed while the grid would not fill the GPU twice over
    int bn = 256;
    while (bn > N) bn >>= 1;
    int dev = 0, sms = 148;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    while (bn > 64 && tiles_m * ((N + bn - 1) / bn) * phases < 2LL * sms) bn >>= 1;
    const CUtensorMapSwizzle sw = KC == 64 ? CU_TENSOR_MAP_SWIZZLE_128B : CU_TENSOR_MAP_SWIZZLE_64B;
    CUtensorMap ta, tb;
    const cuuint64_t adim[4] = {(cuuint64_t)C, (cuuint64_t)W, (cuuint64_t)H, (cuuint64_t)Bimg};
    const cuuint64_t astr[3] = {(cuuint64_t)ld * 2, (cuuint64_t)W * ld * 2, (cuuint64_t)H * W * ld * 2};
    const cuuint32_t abox[4] = {(cuuint32_t)KC, 16, 8, 1};
    const cuuint32_t one[4] = {1, 1, 1, 1};
    if (enc(&ta, CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 4, const_cast<bf16*>(x + off), adim, astr, abox, one,
            CU_TENSOR_MAP_INTERLEAVE_NONE, sw, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
            CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) != CUDA_SUCCESS)
        return false;
    const cuuint64_t bdim[2] = {(cuuint64_t)taps * C, (cuuint64_t)phases * rows_per_phase};
    const cuuint64_t bstr[1] = {(cuuint64_t)taps * C * 2};
    const cuuint32_t bbox[2] = {(cuuint32_t)KC, (cuuint32_t)bn};
    if (enc(&tb, CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 2, const_cast<bf16*>(w), bdim, bstr, bbox, one,
            CU_TENSOR_MAP_INTERLEAVE_NONE, sw, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
            CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) != CUDA_SUCCESS)
        return false;
    UmmaShape sh{H, W, C, taps, (C + KC - 1) / KC, N, rows_per_phase};
    const dim3 grid((unsigned)tiles_m, (unsigned)((N + bn - 1) / bn), (unsigned)phases);
    return KC == 64 ? launch_umma_bn<64>(bn, s, ta, tb, ep, sh, grid) : launch_umma_bn<32>(bn, s, ta, tb, ep, sh, grid);
}

template <int AW, int BN, int BW>
bool launch_wgrad(cudaStream_t s, const CUtensorMap& tx, const CUtensorMap& tg, const EpPartial& ep,
                  const UmmaWgrad& sh, dim3 grid)
{
    constexpr int bytes = WgradSmem<AW, BN, BW>::BYTES;
    static const bool attr = cudaFuncSetAttribute(k_umma_wgrad<AW, BN, BW>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                                  bytes) == cudaSuccess;
    if (!attr) return false;
    k_umma_wgrad<AW, BN, BW><<<grid, 128, bytes, s>>>(tx, tg, ep, sh);
    return cudaGetLastError() == cudaSuccess;
}

template <int AW>
bool launch_wgrad_bn(int bn, cudaStream_t s, const CUtensorMap& tx, const CUtensorMap& tg, const EpPartial& ep,
                     const UmmaWgrad& sh, dim3 grid)
{
    switch (bn) {
    case 32: return launch_wgrad<AW, 32, 32>(s, tx, tg, ep, sh, grid);
    case 64: return launch_wgrad<AW, 64, 64>(s, tx, tg, ep, sh, grid);
    case 128: return launch_wgrad<AW, 128, 64>(s, tx, tg, ep, sh, grid);
    default: return launch_wgrad<AW, 256, 64>(s, tx, tg, ep, sh, grid);
    }
}

// The weight gradient of a 3x3 convolution (k_umma_wgrad) into FP32 partials
// part[split][9 Cin][Cout] (at most part_cap floats): x is the layer input
// (Bimg images H x W, Cin channels at row stride ld from channel off), g the
// pre-activation gradient ([pixels][Cout]).  Returns the number of splits
// written, or 0 when the shapes do not allow it (nothing launched).
int umma_wgrad(cudaStream_t s, const bf16* x, int Bimg, int H, int W, int Cin, int ld, int off, const bf16* g,
               int Cout, float* part, long long part_cap, int g_ld = 0)
{
    // g_ld > 0: the transposed convolution's weight gradient (x the H x W input, g the 2H x 2W output gradient with
    // row stride g_ld; four phases, partials part[split][phase][Cin][Cout])
    const bool up = g_ld > 0;
    if (g_engine != UNET_ENGINE_TCGEN05) return 0;
    if ((Cin % 64 && Cin != 32) || (Cout % 64 && Cout != 32) || W % 16 || H % 4 || ld % 8 || off % 8) return 0;
    umma::EncodeTiledFn enc = umma::tensor_map_encoder();
    if (!enc) return 0;
    const long long Mw = (up ? 1LL : 9LL) * Cin;
    const int phases = up ? 4 : 1;
    const int aw = Cin % 64 ? 32 : 64;  // channels per A block (and per box)
    const int bn = Cout >= 256 ? 256 : (Cout >= 128 ? 128 : Cout);  // 32, 64, 128 or 256
    const int bw = bn == 32 ? 32 : 64;
    const long long tiles = ((Mw + 127) / 128) * ((Cout + bn - 1) / bn);
    const int cpi = (H / 4) * (W / 16);
    const long long chunks = (long long)Bimg * cpi;
    int dev = 0, sms = 148;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    long long sp = (2LL * sms + tiles * phases - 1) / (tiles * phases);
    sp = std::min(sp, std::max(1LL, chunks / 8));
    sp = std::min(sp, (long long)kMaxSplits);
    sp = std::min(sp, part_cap / (phases * Mw * Cout));
    if (sp < 1) return 0;
    const long long cps = (chunks + sp - 1) / sp;
    sp = (chunks + cps - 1) / cps;
    CUtensorMap tx, tg;
    const cuuint32_t abox[4] = {(cuuint32_t)aw, 16, 4, 1};
    const cuuint32_t bbox[4] = {(cuuint32_t)bw, 16, 4, 1};
    const cuuint32_t one[4] = {1, 1, 1, 1};
    const cuuint32_t one5[5] = {1, 1, 1, 1, 1};
    const CUtensorMapSwizzle asw = aw == 64 ? CU_TENSOR_MAP_SWIZZLE_128B : CU_TENSOR_MAP_SWIZZLE_64B;
    const CUtensorMapSwizzle bsw = bw == 64 ? CU_TENSOR_MAP_SWIZZLE_128B : CU_TENSOR_MAP_SWIZZLE_64B;
    const cuuint64_t xdim[4] = {(cuuint64_t)Cin, (cuuint64_t)W, (cuuint64_t)H, (cuuint64_t)Bimg};
    const cuuint64_t xstr[3] = {(cuuint64_t)ld * 2, (cuuint64_t)W * ld * 2, (cuuint64_t)H * W * ld * 2};
    const cuuint64_t gdim[4] = {(cuuint64_t)Cout, (cuuint64_t)W, (cuuint64_t)H, (cuuint64_t)Bimg};
    const cuuint64_t gstr[3] = {(cuuint64_t)Cout * 2, (cuuint64_t)W * Cout * 2, (cuuint64_t)H * W * Cout * 2};
    // the output gradient of a transposed convolution as (channel, x parity, x pair, y parity, image row pair)
    const cuuint64_t udim[5] = {(cuuint64_t)Cout, 2, (cuuint64_t)W, 2, (cuuint64_t)H * Bimg};
    const cuuint64_t ustr[4] = {(cuuint64_t)g_ld * 2, (cuuint64_t)g_ld * 4, (cuuint64_t)W * g_ld * 4,
                                (cuuint64_t)W * g_ld * 8};
    const cuuint32_t ubox[5] = {(cuuint32_t)bw, 1, 16, 1, 4};
    if (enc(&tx, CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 4, const_cast<bf16*>(x + off), xdim, xstr, abox, one,
            CU_TENSOR_MAP_INTERLEAVE_NONE, asw, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
            CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) != CUDA_SUCCESS ||
        (up ? enc(&tg, CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 5, const_cast<bf16*>(g), udim, ustr, ubox, one5,
                  CU_TENSOR_MAP_INTERLEAVE_NONE, bsw, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
                  CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE)
            : enc(&tg, CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 4, const_cast<bf16*>(g), gdim, gstr, bbox, one,
                  CU_TENSOR_MAP_INTERLEAVE_NONE, bsw, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
                  CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE)) != CUDA_SUCCESS)
        return 0;
    UmmaWgrad sh{H, W, Cin, Cout, Mw, cpi, chunks, (int)cps, up ? 1 : 0, (int)sp};
    EpPartial ep{part, Cout, phases * Mw * Cout, Mw * Cout, 0, 0};
    const dim3 grid((unsigned)((Mw + 127) / 128), (unsigned)((Cout + bn - 1) / bn), (unsigned)(sp * phases));
    const bool ok = aw == 64 ? launch_wgrad_bn<64>(bn, s, tx, tg, ep, sh, grid)
                             : launch_wgrad_bn<32>(bn, s, tx, tg, ep, sh, grid);
    return ok ? (int)sp : 0;
}

// conv3x3 (+bias, ReLU) of x (level geometry H x W, Cin channels at ld/off) into y (contiguous Cout).
void conv_fwd(const Ctx& C, int layer, int wtensor, const bf16* x, int H, int W, int Cin, int ld, int off, bf16* y,
              int Cout)
{
    const long long P = (long long)C.L.B * H * W;
    EpAct ep{y, Cout, 0, C.pw(wtensor + 1), 1};
    if (umma_conv(C.s, x, C.L.B, H, W, Cin, ld, off, 9, C.wf(layer), Cout, 1, Cout, ep)) return;
    LdIm2col<BM> la{x, H, W, Cin, ld, off, 9};
    LdRows<BN> lb{C.wf(layer), 9 * Cin, 0};
    gemm(C.s, la, lb, ep, P, Cout, 9 * Cin, 1, 1);
}

// Split-K count of a weight-gradient product (M x N output, K pixels): enough
// CTAs to fill the GPU (about 4 per SM), at least 16 k-tiles per split.
int splits_for(long long M, long long N, long long K)
{
    const long long tiles = ((M + BM - 1) / BM) * ((N + BN - 1) / BN);
    const long long want = (kTargetCtas + tiles - 1) / tiles;
    const long long most = std::max(1LL, K / (16 * BK));
    return (int)std::max(1LL, std::min(want, std::min(most, (long long)kMaxSplits)));
}

// Weight and bias gradients of a 3x3 convolution with input x (ld/off) and
// pre-activation gradient g (contiguous [P][Cout]); dx into dxo (contiguous
// [P][Cin]) unless null.
void conv_bwd(const Ctx& C, int layer, int wtensor, const bf16* x, int H, int W, int Cin, int ld, int off,
              const bf16* g, int Cout, float* grad, bf16* dxo)
{
    const long long P = (long long)C.L.B * H * W;
    float* part = at<float>(C.ws, C.L.part);
    // dW[(tap, ci)][co] = sum_p x[p + tap][ci] g[p][co]
    const long long Mw = 9LL * Cin;
    int sp = umma_wgrad(C.s, x, C.L.B, H, W, Cin, ld, off, g, Cout, part, C.L.part_floats);
    if (!sp) {
        sp = splits_for(Mw, Cout, P);
        LdGatherT<BM> la{x, H, W, Cin, ld, off, 9, 0, 0};
        LdGatherT<BN> lb{g, H, W, Cout, Cout, 0, 1, 0, 0};
        EpPartial ep{part, Cout, Mw * Cout, 0, 0, 0};
        gemm(C.s, la, lb, ep, Mw, Cout, (int)P, sp, 1);
    }
    sum_partials(C.s, part, Mw * Cout, sp, Mw * Cout, grad + C.t[wtensor].off);
    // db[co] = sum_p g[p][co]
    const long long rows = (P + 255) / 256;
    const int nb = (int)((P + rows - 1) / rows);
    k_colsum<<<nb, 256, 0, C.s>>>(g, P, Cout, Cout, 0, rows, part);
    sum_partials(C.s, part, Cout, nb, Cout, grad + C.t[wtensor + 1].off);
    if (dxo) {
        EpAct ep2{dxo, Cin, 0, nullptr, 0};
        if (umma_conv(C.s, g, C.L.B, H, W, Cout, Cout, 0, 9, C.wb(layer), Cin, 1, Cin, ep2)) return;
        LdIm2col<BM> la2{g, H, W, Cout, Cout, 0, 9};
        LdRows<BN> lb2{C.wb(layer), 9 * Cout, 0};
        gemm(C.s, la2, lb2, ep2, P, Cin, 9 * Cout, 1, 1);
    }
}

// Transposed convolution (2x2, stride 2) of x (level l+1 geometry Hs x Ws,
// Cin contiguous) into the first Cout channels of y (level l, row stride ld).
void up_fwd(const Ctx& C, int layer, int wtensor, const bf16* x, int Hs, int Ws, int Cin, bf16* y, int Cout, int ld)
{
    const long long P = (long long)C.L.B * Hs * Ws;
    EpUp ep{y, Hs, Ws, ld, 0, C.pw(wtensor + 1), 0};
    if (umma_conv(C.s, x, C.L.B, Hs, Ws, Cin, Cin, 0, 1, C.wf(layer), Cout, 4, Cout, ep)) return;
    LdIm2col<BM> la{x, Hs, Ws, Cin, Cin, 0, 1};
    LdRows<BN> lb{C.wf(layer), Cin, (long long)Cout * Cin};
    gemm(C.s, la, lb, ep, P, Cout, Cin, 1, 4);
}

// Gradients of the transposed convolution: input x (Hs x Ws, Cin), output
// gradient in the first Cout channels of gy (row stride ld, level l).
void up_bwd(const Ctx& C, int layer, int wtensor, const bf16* x, int Hs, int Ws, int Cin, const bf16* gy, int Cout,
            int ld, float* grad, bf16* dxo)
{
    const long long P = (long long)C.L.B * Hs * Ws;
    float* part = at<float>(C.ws, C.L.part);
    // dW[phase][ci][co] = sum_p x[p][ci] gy[up(p, phase)][co]
    int sp = umma_wgrad(C.s, x, C.L.B, Hs, Ws, Cin, Cin, 0, gy, Cout, part, C.L.part_floats, ld);
    if (!sp) {
        sp = std::max(1, splits_for(Cin, Cout, P) / 4);  // the four phases multiply the CTAs
        LdGatherT<BM> la{x, Hs, Ws, Cin, Cin, 0, 1, 0, 0};
        LdGatherT<BN> lb{gy, Hs, Ws, Cout, ld, 0, 1, 1, 0};
        EpPartial ep{part, Cout, 4LL * Cin * Cout, (long long)Cin * Cout, 0, 0};
        gemm(C.s, la, lb, ep, Cin, Cout, (int)P, sp, 4);
    }
    sum_partials(C.s, part, 4LL * Cin * Cout, sp, 4LL * Cin * Cout,
                                                               grad + C.t[wtensor].off);
    // db[co] = sum over output pixels of gy[..][co]
    const long long Po = 4 * P;
    const long long rows = (Po + 255) / 256;
    const int nb = (int)((Po + rows - 1) / rows);
    k_colsum<<<nb, 256, 0, C.s>>>(gy, Po, Cout, ld, 0, rows, part);
    sum_partials(C.s, part, Cout, nb, Cout, grad + C.t[wtensor + 1].off);
    // dx[p][ci] = sum_(phase, co) gy[up(p, phase)][co] W[phase][ci][co]
    LdUpGather<BM> la2{gy, Hs, Ws, Cout, ld, 0};
    LdRows<BN> lb2{C.wb(layer), 4 * Cout, 0};
    EpAct ep2{dxo, Cin, 0, nullptr, 0};
    gemm(C.s, la2, lb2, ep2, P, Cin, 4 * Cout, 1, 1);
}

}  // namespace
}  // namespace lbm

using namespace lbm;

extern "C" {

lbm_status unet_set_engine(int32_t engine)
{
    if (engine != UNET_ENGINE_MMA_SYNC && engine != UNET_ENGINE_TCGEN05) return LBM_ERR_INVALID_ARG;
    g_engine = engine;
    return LBM_OK;
}

lbm_status unet_get_status(void)
{
    unsigned flag = 0, zero = 0;
    if (cudaDeviceSynchronize() != cudaSuccess ||
        cudaMemcpyFromSymbol(&flag, g_umma_status, sizeof(flag)) != cudaSuccess ||
        cudaMemcpyToSymbol(g_umma_status, &zero, sizeof(zero)) != cudaSuccess)
        return LBM_ERR_CUDA;
    return flag ? LBM_ERR_TIMEOUT : LBM_OK;
}

lbm_status unet_param_layout(int32_t base, int32_t* n_tensors, int64_t* n_params, int64_t* offsets, int64_t* counts)
{
    if (base < 8 || base % 8 || base > 256 || !n_tensors || !n_params) return LBM_ERR_INVALID_ARG;
    const auto t = param_tensors(base);
    *n_tensors = (int32_t)t.size();
    *n_params = t.back().off + t.back().count;
    for (size_t i = 0; i < t.size(); ++i) {
        if (offsets) offsets[i] = t[i].off;
        if (counts) counts[i] = t[i].count;
    }
    return LBM_OK;
}

lbm_status unet_workspace_size(const unet_desc* d, size_t* bytes)
{
    Layout L;
    if (!bytes || !make_layout(d, &L)) return LBM_ERR_INVALID_ARG;
    *bytes = L.total;
    return LBM_OK;
}

lbm_status unet_pack_input(const unet_desc* d, const double* d_u, const uint8_t* d_mask, double scale, uint16_t* d_x,
                           void* stream)
{
    Layout L;
    if (!make_layout(d, &L) || !d_u || !d_mask || !d_x) return LBM_ERR_INVALID_ARG;
    const long long n = (long long)L.B * L.H * L.W;
    k_pack<<<ew_grid(n), 256, 0, static_cast<cudaStream_t>(stream)>>>(d_u, d_mask, L.B, L.H, L.W, (float)scale,
                                                                      reinterpret_cast<bf16*>(d_x));
    return cuda_status(cudaGetLastError());
}

lbm_status unet_prepare_weights(const unet_desc* d, const float* d_params, void* d_ws, void* stream)
{
    Layout L;
    if (!make_layout(d, &L) || !d_params || !d_ws) return LBM_ERR_INVALID_ARG;
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    std::vector<int> taps, cin, cout;
    const auto t = param_tensors(d->base, &taps, &cin, &cout);
    for (size_t i = 0, layer = 0; i + 2 < t.size(); i += 2, ++layer) {
        const bool up = taps[i] == 4;
        k_prep_weights<<<ew_grid(t[i].count), 256, 0, s>>>(d_params + t[i].off, taps[i], cin[i], cout[i], up ? 0 : 1,
                                                           up ? 1 : 0, at<bf16>(d_ws, L.wf[layer]),
                                                           at<bf16>(d_ws, L.wb[layer]));
    }
    if (cudaMemcpyAsync(at<float>(d_ws, L.bias), d_params, sizeof(float) * (size_t)L.n_params,
                        cudaMemcpyDeviceToDevice, s) != cudaSuccess)
        return LBM_ERR_CUDA;
    return cuda_status(cudaGetLastError());
}

lbm_status unet_forward(const unet_desc* d, const uint16_t* d_x, float* d_out, void* d_ws, void* stream)
{
    Layout L;
    if (!make_layout(d, &L) || !d_x || !d_out || !d_ws) return LBM_ERR_INVALID_ARG;
    Ctx C{L, d_ws, static_cast<cudaStream_t>(stream), param_tensors(d->base)};
    const bf16* x = reinterpret_cast<const bf16*>(d_x);
    int tensor = 0, layer = 0;
    const bf16* in = x;
    int cin = UNET_IN_CHANNELS;
    for (int l = 0; l < 4; ++l) {
        bf16* ea = at<bf16>(d_ws, L.ea[l]);
        bf16* eb = at<bf16>(d_ws, L.eb[l]);
        conv_fwd(C, layer++, tensor, in, L.Hl[l], L.Wl[l], cin, cin, 0, ea, L.c[l]);
        tensor += 2;
        conv_fwd(C, layer++, tensor, ea, L.Hl[l], L.Wl[l], L.c[l], L.c[l], 0, eb, L.c[l]);
        tensor += 2;
        if (l < 3) {
            bf16* pool = at<bf16>(d_ws, L.pool[l]);
            k_maxpool<<<ew_grid(L.P[l + 1] * L.c[l] / 8), 256, 0, C.s>>>(eb, L.B, L.Hl[l], L.Wl[l], L.c[l], pool,
                                                                       at<uint8_t>(d_ws, L.arg[l]));
            k_copy_channels<<<ew_grid(L.P[l] * L.c[l] / 8), 256, 0, C.s>>>(eb, L.P[l], L.c[l], at<bf16>(d_ws, L.cat[l]),
                                                                        2 * L.c[l], L.c[l]);
            in = pool;
            cin = L.c[l];
        }
    }
    const bf16* below = at<bf16>(d_ws, L.eb[3]);
    for (int l = 2; l >= 0; --l) {
        bf16* cat = at<bf16>(d_ws, L.cat[l]);
        up_fwd(C, layer++, tensor, below, L.Hl[l + 1], L.Wl[l + 1], L.c[l + 1], cat, L.c[l], 2 * L.c[l]);
        tensor += 2;
        bf16* da = at<bf16>(d_ws, L.da[l]);
        bf16* db = at<bf16>(d_ws, L.db[l]);
        conv_fwd(C, layer++, tensor, cat, L.Hl[l], L.Wl[l], 2 * L.c[l], 2 * L.c[l], 0, da, L.c[l]);
        tensor += 2;
        conv_fwd(C, layer++, tensor, da, L.Hl[l], L.Wl[l], L.c[l], L.c[l], 0, db, L.c[l]);
        tensor += 2;
        below = db;
    }
    float* out = at<float>(d_ws, L.out);
    k_head<<<L.B * L.H, 256, 0, C.s>>>(below, L.W, L.c[0], C.pw(tensor), C.pw(tensor + 1), out);
    if (cudaMemcpyAsync(d_out, out, sizeof(float) * (size_t)L.B * L.H, cudaMemcpyDeviceToDevice, C.s) != cudaSuccess)
        return LBM_ERR_CUDA;
    return cuda_status(cudaGetLastError());
}

lbm_status unet_backward(const unet_desc* d, const uint16_t* d_x, const float* d_target, float* d_loss, float* d_grad,
                         void* d_ws, void* stream)
{
    Layout L;
    if (!make_layout(d, &L) || !d_x || !d_target || !d_loss || !d_grad || !d_ws) return LBM_ERR_INVALID_ARG;
    Ctx C{L, d_ws, static_cast<cudaStream_t>(stream), param_tensors(d->base)};
    const int nt = (int)C.t.size();
    float* gout = at<float>(d_ws, L.gout);
    float* part = at<float>(d_ws, L.part);
    const int rows = L.B * L.H;
    k_mse<<<1, 256, 0, C.s>>>(at<float>(d_ws, L.out), d_target, rows, d_loss, gout);
    // head: tensors nt-2 (w), nt-1 (b)
    bf16* gA = at<bf16>(d_ws, L.gA);
    bf16* gB = at<bf16>(d_ws, L.gB);
    bf16* gC = at<bf16>(d_ws, L.gC);
    const bf16* db0 = at<bf16>(d_ws, L.db[0]);
    k_head_grad<<<rows, 256, 0, C.s>>>(db0, L.W, L.c[0], C.pw(nt - 2), gout, gA, part);
    sum_partials(C.s, part, L.c[0], rows, L.c[0], d_grad + C.t[nt - 2].off);
    k_sum_vector<<<1, 256, 0, C.s>>>(gout, rows, d_grad + C.t[nt - 1].off);
    // decoder, l = 0, 1, 2 (tensors and layers counted from the end)
    int tensor = nt - 2, layer = 16;  // 17 convolution layers, numbered in forward order
    for (int l = 0; l <= 2; ++l) {
        const int Hl = L.Hl[l], Wl = L.Wl[l], c = L.c[l];
        // gA = dL/d(db_l)
        tensor -= 2;  // dec{l}b
        k_relu_grad<<<ew_grid(L.P[l] * c / 8), 256, 0, C.s>>>(gA, c, 0, at<bf16>(d_ws, L.db[l]), gB, L.P[l], c);
        conv_bwd(C, layer--, tensor, at<bf16>(d_ws, L.da[l]), Hl, Wl, c, c, 0, gB, c, d_grad, gA);
        tensor -= 2;  // dec{l}a
        k_relu_grad<<<ew_grid(L.P[l] * c / 8), 256, 0, C.s>>>(gA, c, 0, at<bf16>(d_ws, L.da[l]), gB, L.P[l], c);
        bf16* gcat = at<bf16>(d_ws, L.gcat[l]);
        conv_bwd(C, layer--, tensor, at<bf16>(d_ws, L.cat[l]), Hl, Wl, 2 * c, 2 * c, 0, gB, c, d_grad, gcat);
        tensor -= 2;  // up{l}
        const bf16* below = l == 2 ? at<bf16>(d_ws, L.eb[3]) : at<bf16>(d_ws, L.db[l + 1]);
        up_bwd(C, layer--, tensor, below, L.Hl[l + 1], L.Wl[l + 1], L.c[l + 1], gcat, c, 2 * c, d_grad, gA);
    }
    // encoder, l = 3 .. 0; gA = dL/d(eb_3) on entry
    for (int l = 3; l >= 0; --l) {
        const int Hl = L.Hl[l], Wl = L.Wl[l], c = L.c[l];
        if (l < 3) {  // gA = dL/d(pool_l) -> dL/d(eb_l), plus the skip gradient
            k_maxpool_grad<<<ew_grid(L.P[l] * c / 8), 256, 0, C.s>>>(gA, at<uint8_t>(d_ws, L.arg[l]), L.B, Hl, Wl, c,
                                                                   at<bf16>(d_ws, L.gcat[l]), 2 * c, c, gC);
            std::swap(gA, gC);
        }
        tensor -= 2;  // enc{l}b
        k_relu_grad<<<ew_grid(L.P[l] * c / 8), 256, 0, C.s>>>(gA, c, 0, at<bf16>(d_ws, L.eb[l]), gB, L.P[l], c);
        conv_bwd(C, layer--, tensor, at<bf16>(d_ws, L.ea[l]), Hl, Wl, c, c, 0, gB, c, d_grad, gA);
        tensor -= 2;  // enc{l}a
        k_relu_grad<<<ew_grid(L.P[l] * c / 8), 256, 0, C.s>>>(gA, c, 0, at<bf16>(d_ws, L.ea[l]), gB, L.P[l], c);
        const int cin = l == 0 ? UNET_IN_CHANNELS : L.c[l - 1];
        const bf16* in = l == 0 ? reinterpret_cast<const bf16*>(d_x) : at<bf16>(d_ws, L.pool[l - 1]);
        conv_bwd(C, layer--, tensor, in, Hl, Wl, cin, cin, 0, gB, c, d_grad, l == 0 ? nullptr : gA);
    }
    return cuda_status(cudaGetLastError());
}

lbm_status unet_adam(int64_t n, float* d_params, float* d_m, float* d_v, const float* d_grad, int32_t t, float lr,
                     float beta1, float beta2, float eps, void* stream)
{
    if (n < 1 || t < 1 || !d_params || !d_m || !d_v || !d_grad) return LBM_ERR_INVALID_ARG;
    const float c1 = 1.0f - powf(beta1, (float)t), c2 = 1.0f - powf(beta2, (float)t);
    k_adam_f32<<<ew_grid(n), 256, 0, static_cast<cudaStream_t>(stream)>>>(n, d_params, d_m, d_v, d_grad, lr, beta1,
                                                                          beta2, eps, c1, c2);
    return cuda_status(cudaGetLastError());
}

}  // extern "C"
