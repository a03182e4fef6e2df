// The learned initial guess for the Newton-Krylov base-flow solve: a
// 4-level U-Net (declared in include/nsstab.h; the paper has no network).
//
// Storage: activations in bfloat16, channels innermost ([B][H][W][C]), so
// the channels of one point are one contiguous run; weights as FP32 masters
// (with Adam's moments) plus a bfloat16 copy that the convolutions read;
// every sum in FP32; gradients of activations in FP32 (bfloat16 hi + lo
// planes where a GEMM reads them).
//
// Kernels (one pass each, no im2col buffer):
//   k_conv_gemm<false>  3x3 periodic convolution + bias + ReLU: implicit GEMM
//                       on the tensor cores (BF16 mma.sync, FP32 accumulate)
//   k_conv_gemm<true>   gradient of the input: the same GEMM with the
//                       channels exchanged and the taps mirrored
//   k_conv_bwd_w        gradient of the weights and bias: per tap a GEMM
//                       reduced over points, split over blocks, atomicAdd
//                       into the FP32 gradient
//   k_relu_split        gradient of a ReLU output as bfloat16 hi + lo planes
//   pooling, upsampling with concatenation, their adjoints, the 1x1 output
//   layer, the mean-squared loss and Adam are pointwise kernels.
// The layer sequence and every rounding point follow the oracle's
// definition of the network (the same flat parameter layout).
#include <cuda_bf16.h>

#include <cmath>
#include <cstdint>
#include <initializer_list>
#include <string>
#include <vector>

#include "common.cuh"

namespace nsstab {
namespace {

using bf16 = __nv_bfloat16;
constexpr int kLevels = 4;

struct ConvDesc {
    int ci = 0, co = 0, k = 3;   // k = 3 (3x3) or 1 (the output layer)
    long w_off = 0, b_off = 0;   // offsets into the flat parameter vector
};

// Neighbour (y + dy, x + dx) of point p = (b, y, x) on the periodic
// 2^lh x 2^lw grid.
__device__ __forceinline__ long nbr(long p, int lh, int lw, int dy, int dx) {
    const int W = 1 << lw, H = 1 << lh;
    const int x = (int)(p & (W - 1));
    const int y = (int)((p >> lw) & (H - 1));
    const long b = p >> (lw + lh);
    return (((b << lh) + ((y + dy) & (H - 1))) << lw) + ((x + dx) & (W - 1));
}

// ---------------------------------------------------------------------------
// The three 3x3 convolutions are implicit GEMMs on the tensor cores (BF16
// mma.sync m16n8k16, FP32 accumulation; products of bfloat16 values are
// exact in FP32, so only the order of the FP32 sums differs from a scalar
// loop).  Operands reach shared memory by 16-byte cp.async copies (VEC: all
// channel counts multiples of 8 and 16-byte aligned bases; otherwise plain
// loads), in a ring of pipeline stages, and reach the registers by ldmatrix.
// Every tile row is padded to 40 bf16 (80 bytes), which makes the ldmatrix
// reads of a warp hit 32 distinct banks.
//
// The FP32 gradient of a ReLU output enters as two bfloat16 planes
// (hi = bf16(g), lo = bf16(g - hi), written by k_relu_split), two mma steps
// per fragment: about 16 significant bits of every product, summed in FP32.
//
// The bfloat16 weight copy wt is tap-major, wt[tap][co][ci], so that a tile
// of (output, input) channels of one tap is a set of contiguous rows for
// either GEMM that reads it.
// ---------------------------------------------------------------------------
constexpr int kMmaCo = 32, kMmaK = 16;
constexpr int kStr = 40;            // padded tile row (bf16)
constexpr int kTilePts = 64;        // points per block in the forward and input-gradient GEMMs
constexpr int kRing = 4;            // pipeline depth of those GEMMs

__device__ __forceinline__ void mma_bf16(float* d, uint32_t a0, uint32_t a1, uint32_t a2, uint32_t a3, uint32_t b0,
                                         uint32_t b1) {
    asm volatile("mma.sync.aligned.m16n8k16.row.col.f32.bf16.bf16.f32 {%0,%1,%2,%3}, {%4,%5,%6,%7}, {%8,%9}, "
                 "{%0,%1,%2,%3};"
                 : "+f"(d[0]), "+f"(d[1]), "+f"(d[2]), "+f"(d[3])
                 : "r"(a0), "r"(a1), "r"(a2), "r"(a3), "r"(b0), "r"(b1));
}

__device__ __forceinline__ uint32_t smem_u32(const void* p) {
    return static_cast<uint32_t>(__cvta_generic_to_shared(p));
}
__device__ __forceinline__ void ldsm_x4(uint32_t addr, uint32_t& r0, uint32_t& r1, uint32_t& r2, uint32_t& r3) {
    asm volatile("ldmatrix.sync.aligned.m8n8.x4.shared.b16 {%0,%1,%2,%3}, [%4];"
                 : "=r"(r0), "=r"(r1), "=r"(r2), "=r"(r3)
                 : "r"(addr));
}
__device__ __forceinline__ void ldsm_x4_t(uint32_t addr, uint32_t& r0, uint32_t& r1, uint32_t& r2, uint32_t& r3) {
    asm volatile("ldmatrix.sync.aligned.m8n8.x4.trans.shared.b16 {%0,%1,%2,%3}, [%4];"
                 : "=r"(r0), "=r"(r1), "=r"(r2), "=r"(r3)
                 : "r"(addr));
}
// 16-byte global -> shared copy; src_bytes = 0 writes zeros
__device__ __forceinline__ void cp_async16(uint32_t dst, const void* src, int src_bytes) {
    asm volatile("cp.async.cg.shared.global [%0], [%1], 16, %2;" ::"r"(dst), "l"(src), "r"(src_bytes));
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;"); }
template <int N>
__device__ __forceinline__ void cp_async_wait() {
    asm volatile("cp.async.wait_group %0;" ::"n"(N));
}

// rows x 32 channels of a [row][LD] bfloat16 array (C channels used) into a
// padded tile: row r of the tile is src_row(r) (negative: zeros), channels
// c0 .. c0 + 31 (zeros at and beyond C; VEC copies whole 8-channel groups,
// so channels C .. LD - 1 must hold zeros).  NT threads share the work.
template <bool VEC, int ROWS, int NT, class RowFn>
__device__ __forceinline__ void stage_rows(bf16 (*tile)[kStr], const bf16* __restrict__ base, int C, int LD, int c0,
                                           RowFn src_row) {
    if (VEC) {
#pragma unroll
        for (int i = 0; i < (ROWS * 4 + NT - 1) / NT; ++i) {
            const int f = threadIdx.x + i * NT;
            if (ROWS * 4 % NT != 0 && f >= ROWS * 4) break;
            const int r = f >> 2, g = f & 3;
            const long row = src_row(r);
            const bool ok = row >= 0 && c0 + 8 * g < C;
            cp_async16(smem_u32(&tile[r][8 * g]), ok ? base + row * LD + c0 + 8 * g : base, ok ? 16 : 0);
        }
    } else {
#pragma unroll 4
        for (int i = 0; i < (ROWS * kMmaCo + NT - 1) / NT; ++i) {
            const int f = threadIdx.x + i * NT;
            if (ROWS * kMmaCo % NT != 0 && f >= ROWS * kMmaCo) break;
            const int r = f / kMmaCo, c = f % kMmaCo;
            const long row = src_row(r);
            tile[r][c] = (row >= 0 && c0 + c < C) ? base[row * LD + c0 + c] : __float2bfloat16_rn(0.f);
        }
    }
}

// Forward (BWD = false): out[p][co] = relu(bias[co] + sum_{tap, ci}
//   wt[tap][co][ci] in[nbr(p, tap)][ci]) in bfloat16; rows = points,
//   columns = output channels, reduction = (tap, input channel).
// Input gradient (BWD = true): gin[q][ci] = sum_{tap, co} wt[tap][co][ci]
//   gz[q - tap offset][co] in FP32; rows = points, columns = input channels,
//   reduction = (tap, output channel), A = the gradient's hi and lo planes.
// A block of 4 warps owns 64 points x 32 columns (warp w: points 16 w .. +15,
// all 32 columns); one pipeline stage is one tap and 32 reduction channels.
// VA / VB: 16-byte copies for the A rows (row stride lda) / the weight rows.
template <bool BWD, bool VA, bool VB>
__global__ void __launch_bounds__(128) k_conv_gemm(const bf16* __restrict__ a_hi, const bf16* __restrict__ a_lo,
                                                   const bf16* __restrict__ wt, const float* __restrict__ bias,
                                                   void* __restrict__ out, long P, int lh, int lw, int Ci, int Co,
                                                   int lda) {
    constexpr int NP = BWD ? 2 : 1;   // A planes
    struct Stage {
        bf16 a[NP][kTilePts][kStr];
        bf16 b[kMmaCo][kStr];   // forward: [co][ci]; input gradient: [co][ci] read transposed
    };
    extern __shared__ __align__(16) unsigned char smem[];
    Stage* ring = reinterpret_cast<Stage*>(smem);
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int Ck = BWD ? Co : Ci;   // reduction channels per tap
    const int Cn = BWD ? Ci : Co;   // output columns
    const long pb = (long)blockIdx.x * kTilePts;
    const int n0 = blockIdx.y * kMmaCo;
    const int nck = (Ck + kMmaCo - 1) / kMmaCo;
    const int nst = 9 * nck;
    auto issue = [&](int s) {
        Stage& st = ring[s % kRing];
        const int t = s % 9, kc = (s / 9) * kMmaCo;
        const int dy = BWD ? 1 - t / 3 : t / 3 - 1, dx = BWD ? 1 - t % 3 : t % 3 - 1;
        auto arow = [&](int r) -> long {
            const long p = pb + r;
            return p < P ? nbr(p, lh, lw, dy, dx) : -1;
        };
#pragma unroll
        for (int h = 0; h < NP; ++h) stage_rows<VA, kTilePts, 128>(st.a[h], h ? a_lo : a_hi, Ck, lda, kc, arow);
        if (BWD) {   // rows = output channels kc .. kc + 31 (reduction), columns = input channels
            stage_rows<VB, kMmaCo, 128>(st.b, wt + (long)t * Co * Ci, Ci, Ci, n0, [&](int r) -> long {
                return kc + r < Co ? (long)(kc + r) : -1;
            });
        } else {     // rows = output channels n0 .. n0 + 31 (columns), columns = input channels
            stage_rows<VB, kMmaCo, 128>(st.b, wt + (long)t * Co * Ci, Ci, Ci, kc, [&](int r) -> long {
                return n0 + r < Co ? (long)(n0 + r) : -1;
            });
        }
    };
    float acc[4][4];
#pragma unroll
    for (int j = 0; j < 4; ++j)
#pragma unroll
        for (int r = 0; r < 4; ++r) acc[j][r] = 0.f;
    // ldmatrix: lane = 8 i + r supplies row r of 8x8 matrix i
    const int lr = lane & 7, li = lane >> 3;
    const int a_m = warp * 16 + (li & 1) * 8 + lr, a_k = (li >> 1) * 8;        // A [point][k]
    const int bf_n = (li >> 1) * 8 + lr, bf_k = (li & 1) * 8;                  // forward B [n][k]
    const int bb_k = (li & 1) * 8 + lr, bb_n = (li >> 1) * 8;                  // input-gradient B [k][n]
#pragma unroll
    for (int s = 0; s < kRing - 1; ++s) {
        if (s < nst) issue(s);
        cp_async_commit();
    }
    for (int s = 0; s < nst; ++s) {
        cp_async_wait<kRing - 2>();
        __syncthreads();
        if (s + kRing - 1 < nst) issue(s + kRing - 1);
        cp_async_commit();
        const Stage& st = ring[s % kRing];
#pragma unroll
        for (int k0 = 0; k0 < kMmaCo; k0 += kMmaK) {
            uint32_t a[NP][4];
#pragma unroll
            for (int h = 0; h < NP; ++h) ldsm_x4(smem_u32(&st.a[h][a_m][k0 + a_k]), a[h][0], a[h][1], a[h][2], a[h][3]);
#pragma unroll
            for (int jj = 0; jj < 2; ++jj) {
                uint32_t b0, b1, b2, b3;
                if (BWD)
                    ldsm_x4_t(smem_u32(&st.b[k0 + bb_k][16 * jj + bb_n]), b0, b1, b2, b3);
                else
                    ldsm_x4(smem_u32(&st.b[16 * jj + bf_n][k0 + bf_k]), b0, b1, b2, b3);
#pragma unroll
                for (int h = 0; h < NP; ++h) {
                    mma_bf16(acc[2 * jj], a[h][0], a[h][1], a[h][2], a[h][3], b0, b1);
                    mma_bf16(acc[2 * jj + 1], a[h][0], a[h][1], a[h][2], a[h][3], b2, b3);
                }
            }
        }
    }
    cp_async_wait<0>();
    const int gid = lane >> 2, tig = lane & 3;
#pragma unroll
    for (int j = 0; j < 4; ++j) {
#pragma unroll
        for (int r = 0; r < 4; ++r) {
            const long p = pb + warp * 16 + gid + (r >> 1) * 8;
            const int n = n0 + j * 8 + 2 * tig + (r & 1);
            if (p >= P || n >= Cn) continue;
            if (BWD)
                static_cast<float*>(out)[p * Cn + n] = acc[j][r];
            else
                static_cast<bf16*>(out)[p * Cn + n] = __float2bfloat16_rn(fmaxf(acc[j][r] + bias[n], 0.f));
        }
    }
}
template <bool BWD>
constexpr int conv_gemm_smem() {
    return kRing * ((BWD ? 2 : 1) * kTilePts * kStr + kMmaCo * kStr) * (int)sizeof(bf16);
}

// gw[co][ci][tap] += sum_p gz[p][co] in[nbr(p, tap)][ci]; gb[co] += sum_p gz[p][co]
// on the tensor cores: per tap a GEMM with rows = output channels, columns =
// input channels and the reduction over points.  A block owns 32 x 32
// (output, input) channels, all 9 taps, and a chunk of points (a multiple of
// kWgPts); partial sums go to the gradient by atomicAdd.  A stage holds,
// point-major, the gradient's hi and lo planes and the 9 neighbour rows of
// the input; fragments of both come from ldmatrix.trans.  Warp w owns output
// rows 16 (w & 1) .. +15 and input columns 16 (w >> 1) .. +15 for all 9 taps
// (72 FP32 accumulators a thread).  VA / VB: 16-byte copies for the gradient
// planes / the input rows (row stride ldin).  HALO (grid rows of at least
// kWgPts points, so that a stage's points lie in one row): the stage holds
// the 3 input rows y - 1, y, y + 1 over points x - 1 .. x + kWgPts once,
// and tap (dy, dx) reads them shifted by dx, instead of 9 separate
// neighbour rows per point (2.6x fewer staged bytes).
constexpr int kWgPts = 32;   // points per stage
constexpr int kWgRing = 2;
template <bool HALO>
struct WgStage {
    bf16 ah[kWgPts][kStr], al[kWgPts][kStr];   // [point][co]
    // HALO: [dy + 1][1 + dx + point][ci]; else [tap][point][ci]
    bf16 b[HALO ? 3 : 9][HALO ? kWgPts + 2 : kWgPts][kStr];
};
template <bool HALO>
constexpr int wg_smem() {
    return kWgRing * (int)sizeof(WgStage<HALO>);
}

template <bool VA, bool VB, bool HALO>
__global__ void __launch_bounds__(128) k_conv_bwd_w(const bf16* __restrict__ gzh, const bf16* __restrict__ gzl,
                                                    const bf16* __restrict__ in, float* __restrict__ gw,
                                                    float* __restrict__ gb, long P, int lh, int lw, int Ci, int Co,
                                                    int ldin, long chunk) {
    extern __shared__ __align__(16) unsigned char smem[];
    WgStage<HALO>* ring = reinterpret_cast<WgStage<HALO>*>(smem);
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int ci_tiles = (Ci + kMmaCo - 1) / kMmaCo;
    const int co0 = (blockIdx.x / ci_tiles) * kMmaCo, ci0 = (blockIdx.x % ci_tiles) * kMmaCo;
    const long p0 = blockIdx.y * chunk, p1 = min(P, p0 + chunk);
    const int nst = (int)((p1 - p0 + kWgPts - 1) / kWgPts);
    const int mrow = (warp & 1) * 16, ncol = (warp >> 1) * 16;
    auto issue = [&](int s) {
        WgStage<HALO>& st = ring[s % kWgRing];
        const long ps = p0 + (long)s * kWgPts;
        auto prow = [&](int r) -> long { return ps + r < p1 ? ps + r : -1; };
        stage_rows<VA, kWgPts, 128>(st.ah, gzh, Co, Co, co0, prow);
        stage_rows<VA, kWgPts, 128>(st.al, gzl, Co, Co, co0, prow);
        if (HALO) {
            // every point of the stage is a grid point of one row (the rows
            // hold a multiple of kWgPts points); points past p1 meet a zero
            // gradient, so their input values add nothing
#pragma unroll
            for (int r = 0; r < 3; ++r)
                stage_rows<VB, (HALO ? kWgPts + 2 : kWgPts), 128>(st.b[r], in, Ci, ldin, ci0, [&](int q) -> long {
                    return nbr(ps, lh, lw, r - 1, q - 1);
                });
        } else {
#pragma unroll
            for (int t = 0; t < 9; ++t)
                stage_rows<VB, kWgPts, 128>(st.b[t], in, Ci, ldin, ci0, [&](int r) -> long {
                    return ps + r < p1 ? nbr(ps + r, lh, lw, t / 3 - 1, t % 3 - 1) : -1;
                });
        }
    };
    // ldmatrix.trans row addresses: lane = 8 i + r supplies row r of matrix i
    const int lr = lane & 7, li = lane >> 3;
    const int a_k = (li >> 1) * 8 + lr, a_m = mrow + (li & 1) * 8;   // A^T stored [point][co]
    const int b_k = (li & 1) * 8 + lr, b_n = ncol + (li >> 1) * 8;   // B stored [point][ci]
    float acc[9][2][4];
#pragma unroll
    for (int t = 0; t < 9; ++t)
#pragma unroll
        for (int j = 0; j < 2; ++j)
#pragma unroll
            for (int r = 0; r < 4; ++r) acc[t][j][r] = 0.f;
    float accb = 0.f;   // thread tid < 32 of a ci0 = 0 block: channel co0 + tid
    const bool do_b = ci0 == 0 && threadIdx.x < kMmaCo && co0 + (int)threadIdx.x < Co;
#pragma unroll
    for (int s = 0; s < kWgRing - 1; ++s) {
        if (s < nst) issue(s);
        cp_async_commit();
    }
    for (int s = 0; s < nst; ++s) {
        cp_async_wait<kWgRing - 2>();
        __syncthreads();
        if (s + kWgRing - 1 < nst) issue(s + kWgRing - 1);
        cp_async_commit();
        const WgStage<HALO>& st = ring[s % kWgRing];
        if (do_b)
#pragma unroll 8
            for (int k = 0; k < kWgPts; ++k)
                accb += __bfloat162float(st.ah[k][threadIdx.x]) + __bfloat162float(st.al[k][threadIdx.x]);
#pragma unroll
        for (int k0 = 0; k0 < kWgPts; k0 += kMmaK) {
            uint32_t h0, h1, h2, h3, l0, l1, l2, l3;
            ldsm_x4_t(smem_u32(&st.ah[k0 + a_k][a_m]), h0, h1, h2, h3);
            ldsm_x4_t(smem_u32(&st.al[k0 + a_k][a_m]), l0, l1, l2, l3);
#pragma unroll
            for (int t = 0; t < 9; ++t) {
                uint32_t b00, b01, b10, b11;
                const bf16* brow = HALO ? &st.b[t / 3][k0 + b_k + t % 3][b_n] : &st.b[t][k0 + b_k][b_n];
                ldsm_x4_t(smem_u32(brow), b00, b01, b10, b11);
                mma_bf16(acc[t][0], h0, h1, h2, h3, b00, b01);
                mma_bf16(acc[t][0], l0, l1, l2, l3, b00, b01);
                mma_bf16(acc[t][1], h0, h1, h2, h3, b10, b11);
                mma_bf16(acc[t][1], l0, l1, l2, l3, b10, b11);
            }
        }
    }
    cp_async_wait<0>();
    const int gid = lane >> 2, tig = lane & 3;
#pragma unroll
    for (int t = 0; t < 9; ++t) {
#pragma unroll
        for (int j = 0; j < 2; ++j) {
#pragma unroll
            for (int r = 0; r < 4; ++r) {
                const int co = co0 + mrow + gid + (r >> 1) * 8;
                const int ci = ci0 + ncol + j * 8 + 2 * tig + (r & 1);
                if (co < Co && ci < Ci) atomicAdd(&gw[((long)co * Ci + ci) * 9 + t], acc[t][j][r]);
            }
        }
    }
    if (do_b) atomicAdd(&gb[co0 + threadIdx.x], accb);
}

// x [B][C][H][W] FP32 -> [B][H][W][LD] bfloat16, channels C .. LD - 1 zero
__global__ void k_to_nhwc(const float* __restrict__ x, bf16* __restrict__ out, long P, int HW, int C, int LD) {
    for (long e = blockIdx.x * (long)blockDim.x + threadIdx.x; e < P * LD; e += (long)gridDim.x * blockDim.x) {
        const long p = e / LD;
        const int c = (int)(e % LD);
        const long b = p / HW, s = p % HW;
        out[e] = (c < C) ? __float2bfloat16_rn(x[(b * C + c) * HW + s]) : __float2bfloat16_rn(0.f);
    }
}

// 2x2 mean of [B][H][W][C] -> [B][H/2][W/2][C], rounded to bfloat16
__global__ void k_pool(const bf16* __restrict__ in, bf16* __restrict__ out, long Pout, int Ho, int Wo, int C) {
    for (long e = blockIdx.x * (long)blockDim.x + threadIdx.x; e < Pout * C; e += (long)gridDim.x * blockDim.x) {
        const long p = e / C;
        const int c = (int)(e % C);
        const int x = (int)(p % Wo);
        const long r = p / Wo;
        const int y = (int)(r % Ho);
        const long b = r / Ho;
        const int W = 2 * Wo;
        const long i00 = ((b * 2 * Ho + 2 * y) * W + 2 * x) * C + c;
        const float s = __bfloat162float(in[i00]) + __bfloat162float(in[i00 + C]) +
                        __bfloat162float(in[i00 + (long)W * C]) + __bfloat162float(in[i00 + (long)W * C + C]);
        out[e] = __float2bfloat16_rn(0.25f * s);
    }
}

// out[b][y][x] = (low[b][y/2][x/2][0..C1), skip[b][y][x][0..C2))
__global__ void k_up_cat(const bf16* __restrict__ low, const bf16* __restrict__ skip, bf16* __restrict__ out,
                         long P, int H, int W, int C1, int C2) {
    const int C = C1 + C2;
    for (long e = blockIdx.x * (long)blockDim.x + threadIdx.x; e < P * C; e += (long)gridDim.x * blockDim.x) {
        const long p = e / C;
        const int c = (int)(e % C);
        if (c < C1) {
            const int x = (int)(p % W);
            const long r = p / W;
            const int y = (int)(r % H);
            const long b = r / H;
            out[e] = low[((b * (H / 2) + y / 2) * (W / 2) + x / 2) * C1 + c];
        } else {
            out[e] = skip[p * C2 + (c - C1)];
        }
    }
}

// adjoint of k_up_cat: glow[q][c] = sum over the 2x2 children of g[.][c];
// gskip[p][c] = g[p][C1 + c]
__global__ void k_up_cat_bwd(const float* __restrict__ g, float* __restrict__ glow, float* __restrict__ gskip,
                             long Plow, int Hl, int Wl, int C1, int C2) {
    const int C = C1 + C2, W = 2 * Wl;
    for (long e = blockIdx.x * (long)blockDim.x + threadIdx.x; e < Plow * C; e += (long)gridDim.x * blockDim.x) {
        const long q = e / C;
        const int c = (int)(e % C);
        const int x = (int)(q % Wl);
        const long r = q / Wl;
        const int y = (int)(r % Hl);
        const long b = r / Hl;
        const long p00 = (b * 2 * Hl + 2 * y) * W + 2 * x;
        const long ps[4] = {p00, p00 + 1, p00 + W, p00 + W + 1};
        if (c < C1) {
            float s = 0.f;
            for (int k = 0; k < 4; ++k) s += g[ps[k] * C + c];
            glow[q * C1 + c] = s;
        } else {
            for (int k = 0; k < 4; ++k) gskip[ps[k] * C2 + (c - C1)] = g[ps[k] * C + c];
        }
    }
}

// adjoint of k_pool plus the skip gradient: g[p][c] = glow[parent][c] / 4 + gskip[p][c]
__global__ void k_pool_bwd_add(const float* __restrict__ glow, const float* __restrict__ gskip, float* __restrict__ g,
                               long P, int H, int W, int C) {
    for (long e = blockIdx.x * (long)blockDim.x + threadIdx.x; e < P * C; e += (long)gridDim.x * blockDim.x) {
        const long p = e / C;
        const int c = (int)(e % C);
        const int x = (int)(p % W);
        const long r = p / W;
        const int y = (int)(r % H);
        const long b = r / H;
        g[e] = 0.25f * glow[((b * (H / 2) + y / 2) * (W / 2) + x / 2) * C + c] + gskip[e];
    }
}

// g *= (a > 0): the ReLU derivative from the stored activation
// gradient of a ReLU output as the two bfloat16 planes the convolution
// GEMMs read: v = g where the activation is positive, else 0; hi = bf16(v),
// lo = bf16(v - hi)
__global__ void k_relu_split(const float* __restrict__ g, const bf16* __restrict__ a, bf16* __restrict__ hi,
                             bf16* __restrict__ lo, long n) {
    for (long e = blockIdx.x * (long)blockDim.x + threadIdx.x; e < n; e += (long)gridDim.x * blockDim.x) {
        const float v = (__bfloat162float(a[e]) > 0.f) ? g[e] : 0.f;
        const bf16 h = __float2bfloat16_rn(v);
        hi[e] = h;
        lo[e] = __float2bfloat16_rn(v - __bfloat162float(h));
    }
}

// y[p] = b + sum_c w[c] h[p][c]
__global__ void k_out_fwd(const bf16* __restrict__ h, const bf16* __restrict__ w, const float* __restrict__ b,
                          float* __restrict__ y, long P, int C) {
    for (long p = blockIdx.x * (long)blockDim.x + threadIdx.x; p < P; p += (long)gridDim.x * blockDim.x) {
        float s = b[0];
        for (int c = 0; c < C; ++c) s = fmaf(__bfloat162float(w[c]), __bfloat162float(h[p * C + c]), s);
        y[p] = s;
    }
}

// gy = 2 (y - t) / P; partial[block] = sum (y - t)^2 (FP64)
__global__ void k_mse(const float* __restrict__ y, const float* __restrict__ t, float* __restrict__ gy,
                      double* __restrict__ partial, long P) {
    double acc = 0.0;
    const float sc = 2.0f / (float)P;
    for (long p = blockIdx.x * (long)blockDim.x + threadIdx.x; p < P; p += (long)gridDim.x * blockDim.x) {
        const float d = y[p] - t[p];
        gy[p] = sc * d;
        acc += (double)d * (double)d;
    }
    for (int o = 16; o > 0; o >>= 1) acc += __shfl_down_sync(0xffffffffu, acc, o);
    __shared__ double red[32];
    if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = acc;
    __syncthreads();
    if (threadIdx.x < 32) {
        acc = (threadIdx.x < (blockDim.x >> 5)) ? red[threadIdx.x] : 0.0;
        for (int o = 16; o > 0; o >>= 1) acc += __shfl_down_sync(0xffffffffu, acc, o);
        if (threadIdx.x == 0) partial[blockIdx.x] = acc;
    }
}

// output layer backward: gh[p][c] = w[c] gy[p]; gw[c] += sum_p gy[p] h[p][c]; gb += sum_p gy[p]
// blockDim.x = 256 points, one block per chunk; thread c < C of the block's
// second phase reduces channel c over the chunk.
__global__ void k_out_bwd(const float* __restrict__ gy, const bf16* __restrict__ h, const bf16* __restrict__ w,
                          float* __restrict__ gh, float* __restrict__ gw, float* __restrict__ gb, long P, int C) {
    const long p0 = blockIdx.x * 256L;
    for (int e = threadIdx.x; e < 256 * C; e += blockDim.x) {
        const long p = p0 + e / C;
        const int c = e % C;
        if (p < P) gh[p * C + c] = __bfloat162float(w[c]) * gy[p];
    }
    for (int c = threadIdx.x; c <= C; c += blockDim.x) {
        float s = 0.f;
        for (long p = p0; p < min(P, p0 + 256); ++p) s += (c < C) ? gy[p] * __bfloat162float(h[p * C + c]) : gy[p];
        atomicAdd(c < C ? &gw[c] : gb, s);
    }
}

// where the bfloat16 copy of flat parameter i lives: the 3x3 weights
// [co][ci][tap] of each convolution tap-major as [tap][co][ci] at the same
// offset; biases and the output layer in place
struct WtMap {
    int n = 0;
    long off[16];
    int ci[16], co[16];
};
__device__ __forceinline__ long wt_index(const WtMap& m, long i) {
    for (int c = 0; c < m.n; ++c) {
        const long j = i - m.off[c];
        const long sz = 9L * m.ci[c] * m.co[c];
        if (j >= 0 && j < sz) {
            const int t = (int)(j % 9);
            const long oc = j / 9;   // co * ci + ci_
            return m.off[c] + (long)t * m.co[c] * m.ci[c] + oc;
        }
    }
    return i;
}

__global__ void k_adam(float* __restrict__ th, const float* __restrict__ g, float* __restrict__ m, float* __restrict__ v,
                       bf16* __restrict__ wt, WtMap map, long n, float lr, float b1, float b2, float eps, float c1,
                       float c2) {
    for (long i = blockIdx.x * (long)blockDim.x + threadIdx.x; i < n; i += (long)gridDim.x * blockDim.x) {
        const float gi = g[i];
        const float mi = b1 * m[i] + (1.f - b1) * gi;
        const float vi = b2 * v[i] + (1.f - b2) * gi * gi;
        m[i] = mi;
        v[i] = vi;
        const float t = th[i] - lr * (mi / c1) / (sqrtf(vi / c2) + eps);
        th[i] = t;
        wt[wt_index(map, i)] = __float2bfloat16_rn(t);
    }
}

__global__ void k_to_bf16(const float* __restrict__ a, bf16* __restrict__ wt, WtMap map, long n) {
    for (long i = blockIdx.x * (long)blockDim.x + threadIdx.x; i < n; i += (long)gridDim.x * blockDim.x)
        wt[wt_index(map, i)] = __float2bfloat16_rn(a[i]);
}

unsigned grid_for(long n, int threads) {
    const long b = (n + threads - 1) / threads;
    return (unsigned)std::max<long>(1, std::min<long>(b, 152L * 32));
}

}  // namespace
}  // namespace nsstab

using namespace nsstab;

struct nsstab_unet {
    int in_ch = 0, width = 0, H = 0, W = 0, lh = 0, lw = 0, maxB = 0;
    int ldx = 0;                  // channel stride of the bfloat16 input (in_ch rounded up to 8)
    cudaStream_t stream = nullptr;
    long count = 0;
    int step = 0;
    std::vector<ConvDesc> conv;   // 14 convolutions in forward order, then the output layer
    std::vector<void*> allocs;
    float *theta = nullptr, *grad = nullptr, *m = nullptr, *v = nullptr;
    bf16* wt = nullptr;           // bfloat16 weights, 3x3 convolutions tap-major
    WtMap map;
    bf16 *gzh = nullptr, *gzl = nullptr;   // a ReLU output's gradient as bf16 hi + lo planes
    bf16* x = nullptr;
    bf16* act[14] = {};           // ReLU outputs of the 14 convolutions
    bf16* pool[kLevels - 1] = {};
    bf16* cat[kLevels - 1] = {};  // decoder inputs, by level
    float* y = nullptr;
    float* gy = nullptr;
    float *g0 = nullptr, *g1 = nullptr;   // gradient ping-pong
    float* gskip[kLevels - 1] = {};
    float* glow = nullptr;
    double* partial = nullptr;
    double* partial_host = nullptr;

    template <class P> int alloc(P** p, size_t count_) {
        void* q = nullptr;
        const cudaError_t e = cudaMalloc(&q, std::max<size_t>(count_, 1) * sizeof(P));
        if (e != cudaSuccess) {
            set_error(std::string("unet: cudaMalloc: ") + cudaGetErrorString(e));
            return e == cudaErrorMemoryAllocation ? NSSTAB_ERR_OUT_OF_MEMORY : NSSTAB_ERR_CUDA;
        }
        allocs.push_back(q);
        *p = static_cast<P*>(q);
        return NSSTAB_OK;
    }
    ~nsstab_unet() {
        if (stream) cudaStreamSynchronize(stream);
        for (void* p : allocs) cudaFree(p);
        if (partial_host) cudaFreeHost(partial_host);
    }
    int c(int l) const { return width << l; }
    int h(int l) const { return H >> l; }
    int w(int l) const { return W >> l; }
};

namespace {

constexpr int kRedBlocksU = 128;

std::vector<ConvDesc> make_layout(int in_ch, int width, long* count) {
    std::vector<ConvDesc> v;
    long off = 0;
    auto add = [&](int ci, int co, int k) {
        ConvDesc d;
        d.ci = ci;
        d.co = co;
        d.k = k;
        d.w_off = off;
        off += (long)co * ci * k * k;
        d.b_off = off;
        off += co;
        v.push_back(d);
    };
    int ci = in_ch;
    for (int l = 0; l < kLevels; ++l) {
        add(ci, width << l, 3);
        add(width << l, width << l, 3);
        ci = width << l;
    }
    for (int l = kLevels - 2; l >= 0; --l) {
        add((width << (l + 1)) + (width << l), width << l, 3);
        add(width << l, width << l, 3);
    }
    add(width, 1, 1);
    *count = off;
    return v;
}

// indices into conv[] / act[]: encoder level l conv s (0 = a, 1 = b) and
// decoder level l conv s
int enc_id(int l, int s) { return 2 * l + s; }
int dec_id(int l, int s) { return 2 * kLevels + 2 * (kLevels - 2 - l) + s; }

bool al16(const void* p) { return reinterpret_cast<uintptr_t>(p) % 16 == 0; }

using GemmFn = void (*)(const bf16*, const bf16*, const bf16*, const float*, void*, long, int, int, int, int, int);
using WgradFn = void (*)(const bf16*, const bf16*, const bf16*, float*, float*, long, int, int, int, int, int, long);
template <bool BWD>
GemmFn pick_gemm(bool va, bool vb) {
    return va ? (vb ? k_conv_gemm<BWD, true, true> : k_conv_gemm<BWD, true, false>)
              : (vb ? k_conv_gemm<BWD, false, true> : k_conv_gemm<BWD, false, false>);
}
template <bool HALO>
WgradFn pick_wgrad(bool va, bool vb) {
    return va ? (vb ? k_conv_bwd_w<true, true, HALO> : k_conv_bwd_w<true, false, HALO>)
              : (vb ? k_conv_bwd_w<false, true, HALO> : k_conv_bwd_w<false, false, HALO>);
}

// conv id on input rows `in` of stride lda (its input channels, or the
// padded stride of the network input)
int conv_fwd(nsstab_unet* n, int id, const bf16* in, int lda, int l, int B) {
    const ConvDesc& d = n->conv[id];
    const long P = (long)B * n->h(l) * n->w(l);
    const dim3 g((unsigned)((P + kTilePts - 1) / kTilePts), (unsigned)((d.co + kMmaCo - 1) / kMmaCo));
    const bf16* w = n->wt + d.w_off;
    const GemmFn k = pick_gemm<false>(lda % 8 == 0 && al16(in), d.ci % 8 == 0 && al16(w));
    k<<<g, 128, conv_gemm_smem<false>(), n->stream>>>(in, nullptr, w, n->theta + d.b_off, n->act[id], P, n->lh - l,
                                                      n->lw - l, d.ci, d.co, lda);
    NS_LAUNCH_CHECK();
    return NSSTAB_OK;
}

// gradient g (of conv id's ReLU output) -> weight/bias gradients and, when
// gin is not null, the gradient of the conv's input (rows `in`, stride ldin)
int conv_bwd(nsstab_unet* n, int id, const bf16* in, int ldin, const float* g, float* gin, int l, int B) {
    const ConvDesc& d = n->conv[id];
    const long P = (long)B * n->h(l) * n->w(l);
    k_relu_split<<<grid_for(P * d.co, 256), 256, 0, n->stream>>>(g, n->act[id], n->gzh, n->gzl, P * d.co);
    NS_LAUNCH_CHECK();
    const bool vz = d.co % 8 == 0 && al16(n->gzh) && al16(n->gzl);
    // about three blocks per SM in all, each chunk a whole number of stages
    const long tiles = (long)((d.co + kMmaCo - 1) / kMmaCo) * ((d.ci + kMmaCo - 1) / kMmaCo);
    const long nchunk = std::max<long>(1, 3 * 152 / tiles);
    const long chunk = std::max<long>(4 * kWgPts, ((P + nchunk - 1) / nchunk + kWgPts - 1) / kWgPts * kWgPts);
    const dim3 gw((unsigned)tiles, (unsigned)((P + chunk - 1) / chunk));
    const bool vin = ldin % 8 == 0 && al16(in);
    const bool halo = (1L << (n->lw - l)) >= kWgPts;   // a stage's points lie in one grid row
    const WgradFn kw = halo ? pick_wgrad<true>(vz, vin) : pick_wgrad<false>(vz, vin);
    kw<<<gw, 128, halo ? wg_smem<true>() : wg_smem<false>(), n->stream>>>(
        n->gzh, n->gzl, in, n->grad + d.w_off, n->grad + d.b_off, P, n->lh - l, n->lw - l, d.ci, d.co, ldin, chunk);
    NS_LAUNCH_CHECK();
    if (gin) {
        const dim3 gd((unsigned)((P + kTilePts - 1) / kTilePts), (unsigned)((d.ci + kMmaCo - 1) / kMmaCo));
        const bf16* w = n->wt + d.w_off;
        const GemmFn kd = pick_gemm<true>(vz, d.ci % 8 == 0 && al16(w));
        kd<<<gd, 128, conv_gemm_smem<true>(), n->stream>>>(n->gzh, n->gzl, w, nullptr, gin, P, n->lh - l, n->lw - l,
                                                           d.ci, d.co, d.co);
        NS_LAUNCH_CHECK();
    }
    return NSSTAB_OK;
}

int forward(nsstab_unet* n, const float* x, int B) {
    const long P0 = (long)B * n->H * n->W;
    k_to_nhwc<<<grid_for(P0 * n->ldx, 256), 256, 0, n->stream>>>(x, n->x, P0, n->H * n->W, n->in_ch, n->ldx);
    NS_LAUNCH_CHECK();
    const bf16* h = n->x;
    for (int l = 0; l < kLevels; ++l) {
        NS_TRY(conv_fwd(n, enc_id(l, 0), h, l == 0 ? n->ldx : n->c(l - 1), l, B));
        NS_TRY(conv_fwd(n, enc_id(l, 1), n->act[enc_id(l, 0)], n->c(l), l, B));
        h = n->act[enc_id(l, 1)];
        if (l < kLevels - 1) {
            const long Po = (long)B * n->h(l + 1) * n->w(l + 1);
            k_pool<<<grid_for(Po * n->c(l), 256), 256, 0, n->stream>>>(h, n->pool[l], Po, n->h(l + 1), n->w(l + 1),
                                                                       n->c(l));
            NS_LAUNCH_CHECK();
            h = n->pool[l];
        }
    }
    for (int l = kLevels - 2; l >= 0; --l) {
        const long P = (long)B * n->h(l) * n->w(l);
        k_up_cat<<<grid_for(P * (n->c(l + 1) + n->c(l)), 256), 256, 0, n->stream>>>(
            h, n->act[enc_id(l, 1)], n->cat[l], P, n->h(l), n->w(l), n->c(l + 1), n->c(l));
        NS_LAUNCH_CHECK();
        NS_TRY(conv_fwd(n, dec_id(l, 0), n->cat[l], n->c(l + 1) + n->c(l), l, B));
        NS_TRY(conv_fwd(n, dec_id(l, 1), n->act[dec_id(l, 0)], n->c(l), l, B));
        h = n->act[dec_id(l, 1)];
    }
    const ConvDesc& o = n->conv.back();
    k_out_fwd<<<grid_for(P0, 256), 256, 0, n->stream>>>(h, n->wt + o.w_off, n->theta + o.b_off, n->y, P0, n->c(0));
    NS_LAUNCH_CHECK();
    return NSSTAB_OK;
}

int backward(nsstab_unet* n, const float* target, int B, double* loss) {
    const long P0 = (long)B * n->H * n->W;
    NS_CUDA(cudaMemsetAsync(n->grad, 0, n->count * sizeof(float), n->stream));
    k_mse<<<kRedBlocksU, 256, 0, n->stream>>>(n->y, target, n->gy, n->partial, P0);
    NS_LAUNCH_CHECK();
    NS_CUDA(cudaMemcpyAsync(n->partial_host, n->partial, kRedBlocksU * sizeof(double), cudaMemcpyDeviceToHost,
                            n->stream));
    const ConvDesc& o = n->conv.back();
    k_out_bwd<<<(unsigned)((P0 + 255) / 256), 256, 0, n->stream>>>(n->gy, n->act[dec_id(0, 1)], n->wt + o.w_off, n->g0,
                                                                   n->grad + o.w_off, n->grad + o.b_off, P0, n->c(0));
    NS_LAUNCH_CHECK();
    float* g = n->g0;      // gradient of the current layer's output
    float* t = n->g1;      // its input's gradient
    for (int l = 0; l < kLevels - 1; ++l) {
        NS_TRY(conv_bwd(n, dec_id(l, 1), n->act[dec_id(l, 0)], n->c(l), g, t, l, B));
        std::swap(g, t);
        NS_TRY(conv_bwd(n, dec_id(l, 0), n->cat[l], n->c(l + 1) + n->c(l), g, t, l, B));
        std::swap(g, t);
        // g: gradient of cat[l]; split into the level below and the skip
        const long Pl = (long)B * n->h(l + 1) * n->w(l + 1);
        k_up_cat_bwd<<<grid_for(Pl * (n->c(l + 1) + n->c(l)), 256), 256, 0, n->stream>>>(
            g, n->glow, n->gskip[l], Pl, n->h(l + 1), n->w(l + 1), n->c(l + 1), n->c(l));
        NS_LAUNCH_CHECK();
        const long Pn = Pl * n->c(l + 1);
        NS_CUDA(cudaMemcpyAsync(g, n->glow, Pn * sizeof(float), cudaMemcpyDeviceToDevice, n->stream));
    }
    for (int l = kLevels - 1; l >= 0; --l) {
        if (l < kLevels - 1) {
            const long P = (long)B * n->h(l) * n->w(l);
            k_pool_bwd_add<<<grid_for(P * n->c(l), 256), 256, 0, n->stream>>>(g, n->gskip[l], t, P, n->h(l), n->w(l),
                                                                              n->c(l));
            NS_LAUNCH_CHECK();
            std::swap(g, t);
        }
        NS_TRY(conv_bwd(n, enc_id(l, 1), n->act[enc_id(l, 0)], n->c(l), g, t, l, B));
        std::swap(g, t);
        const bf16* in = (l == 0) ? n->x : n->pool[l - 1];
        NS_TRY(conv_bwd(n, enc_id(l, 0), in, l == 0 ? n->ldx : n->c(l - 1), g, l == 0 ? nullptr : t, l, B));
        std::swap(g, t);
    }
    NS_CUDA(cudaStreamSynchronize(n->stream));
    double s = 0.0;
    for (int b = 0; b < kRedBlocksU; ++b) s += n->partial_host[b];
    *loss = s / (double)P0;
    return NSSTAB_OK;
}

int check_batch(nsstab_unet* n, int B, const void* a, const void* b) {
    if (!n || !a || !b) {
        set_error("unet: null argument");
        return NSSTAB_ERR_INVALID_ARG;
    }
    if (B < 1 || B > n->maxB) {
        set_error("unet: batch must be in [1, max_batch]");
        return NSSTAB_ERR_INVALID_ARG;
    }
    return NSSTAB_OK;
}

}  // namespace

extern "C" {

long unet_param_count(int in_ch, int width) {
    if (in_ch < 1 || width < 1) return -1;
    long c = 0;
    make_layout(in_ch, width, &c);
    return c;
}

int unet_create(int in_ch, int width, int ny, int nx, int max_batch, void* stream, nsstab_unet** out) {
    if (!out) {
        set_error("unet_create: null argument");
        return NSSTAB_ERR_INVALID_ARG;
    }
    *out = nullptr;
    const int q = 1 << (kLevels - 1);
    if (in_ch < 1 || in_ch > 64 || width < 1 || width > 256 || max_batch < 1 || ny < q || nx < q ||
        !is_pow2(ny) || !is_pow2(nx) || (long)ny * nx * max_batch > (1L << 28)) {
        set_error("unet_create: need 1 <= in_ch <= 64, 1 <= width <= 256, max_batch >= 1, ny and nx powers of two "
                  ">= 8, max_batch*ny*nx <= 2^28");
        return NSSTAB_ERR_INVALID_ARG;
    }
    bool attr_ok = true;
    for (int va = 0; va < 2; ++va)
        for (int vb = 0; vb < 2; ++vb) {
            attr_ok = attr_ok &&
                      cudaFuncSetAttribute(pick_wgrad<false>(va, vb), cudaFuncAttributeMaxDynamicSharedMemorySize,
                                           wg_smem<false>()) == cudaSuccess &&
                      cudaFuncSetAttribute(pick_wgrad<true>(va, vb), cudaFuncAttributeMaxDynamicSharedMemorySize,
                                           wg_smem<true>()) == cudaSuccess &&
                      cudaFuncSetAttribute(pick_gemm<true>(va, vb), cudaFuncAttributeMaxDynamicSharedMemorySize,
                                           conv_gemm_smem<true>()) == cudaSuccess;
        }
    if (!attr_ok) {
        set_error("unet_create: cudaFuncSetAttribute failed");
        return NSSTAB_ERR_CUDA;
    }
    nsstab_unet* n = new nsstab_unet();
    n->in_ch = in_ch;
    n->ldx = (in_ch + 7) / 8 * 8;
    n->width = width;
    n->H = ny;
    n->W = nx;
    n->lh = ilog2(ny);
    n->lw = ilog2(nx);
    n->maxB = max_batch;
    n->stream = (cudaStream_t)stream;
    n->conv = make_layout(in_ch, width, &n->count);
    for (const ConvDesc& d : n->conv)
        if (d.k == 3) {
            n->map.off[n->map.n] = d.w_off;
            n->map.ci[n->map.n] = d.ci;
            n->map.co[n->map.n] = d.co;
            ++n->map.n;
        }
    const long B = max_batch;
    int rc = NSSTAB_OK;
    auto A = [&](int r) {
        if (rc == NSSTAB_OK) rc = r;
    };
    A(n->alloc(&n->theta, n->count));
    A(n->alloc(&n->grad, n->count));
    A(n->alloc(&n->m, n->count));
    A(n->alloc(&n->v, n->count));
    A(n->alloc(&n->wt, n->count));
    A(n->alloc(&n->x, B * ny * nx * n->ldx));
    for (int l = 0; l < kLevels; ++l) {
        const long P = B * n->h(l) * n->w(l);
        A(n->alloc(&n->act[enc_id(l, 0)], P * n->c(l)));
        A(n->alloc(&n->act[enc_id(l, 1)], P * n->c(l)));
        if (l < kLevels - 1) {
            A(n->alloc(&n->act[dec_id(l, 0)], P * n->c(l)));
            A(n->alloc(&n->act[dec_id(l, 1)], P * n->c(l)));
            A(n->alloc(&n->pool[l], B * n->h(l + 1) * n->w(l + 1) * n->c(l)));
            A(n->alloc(&n->cat[l], P * (n->c(l + 1) + n->c(l))));
            A(n->alloc(&n->gskip[l], P * n->c(l)));
        }
    }
    long gmax = 0;
    for (int l = 0; l < kLevels; ++l) {
        const long P = B * n->h(l) * n->w(l);
        gmax = std::max(gmax, P * (n->c(l) + (l + 1 < kLevels ? n->c(l + 1) : 0)));
        gmax = std::max(gmax, P * (long)(l == 0 ? std::max(in_ch, n->c(0)) : n->c(l - 1)));
    }
    A(n->alloc(&n->gzh, gmax));
    A(n->alloc(&n->gzl, gmax));
    A(n->alloc(&n->g0, gmax));
    A(n->alloc(&n->g1, gmax));
    A(n->alloc(&n->glow, gmax));
    A(n->alloc(&n->y, B * ny * nx));
    A(n->alloc(&n->gy, B * ny * nx));
    A(n->alloc(&n->partial, kRedBlocksU));
    if (rc == NSSTAB_OK && cudaMallocHost((void**)&n->partial_host, kRedBlocksU * sizeof(double)) != cudaSuccess) {
        set_error("unet_create: cudaMallocHost failed");
        rc = NSSTAB_ERR_OUT_OF_MEMORY;
    }
    for (void* z : {(void*)n->theta, (void*)n->m, (void*)n->v})
        if (rc == NSSTAB_OK && cudaMemsetAsync(z, 0, n->count * sizeof(float), n->stream) != cudaSuccess)
            rc = NSSTAB_ERR_CUDA;
    if (rc == NSSTAB_OK && cudaMemsetAsync(n->wt, 0, n->count * sizeof(bf16), n->stream) != cudaSuccess)
        rc = NSSTAB_ERR_CUDA;
    if (rc != NSSTAB_OK) {
        delete n;
        return rc;
    }
    *out = n;
    return NSSTAB_OK;
}

void unet_destroy(nsstab_unet* net) { delete net; }

int unet_set_params(nsstab_unet* net, const float* theta) {
    if (!net || !theta) {
        set_error("unet_set_params: null argument");
        return NSSTAB_ERR_INVALID_ARG;
    }
    NS_CUDA(cudaMemcpyAsync(net->theta, theta, net->count * sizeof(float), cudaMemcpyDeviceToDevice, net->stream));
    NS_CUDA(cudaMemsetAsync(net->m, 0, net->count * sizeof(float), net->stream));
    NS_CUDA(cudaMemsetAsync(net->v, 0, net->count * sizeof(float), net->stream));
    net->step = 0;
    k_to_bf16<<<grid_for(net->count, 256), 256, 0, net->stream>>>(net->theta, net->wt, net->map, net->count);
    NS_LAUNCH_CHECK();
    return NSSTAB_OK;
}

int unet_get_params(nsstab_unet* net, float* theta) {
    if (!net || !theta) {
        set_error("unet_get_params: null argument");
        return NSSTAB_ERR_INVALID_ARG;
    }
    NS_CUDA(cudaMemcpyAsync(theta, net->theta, net->count * sizeof(float), cudaMemcpyDeviceToDevice, net->stream));
    return NSSTAB_OK;
}

int unet_forward(nsstab_unet* net, const float* x, int batch, float* y) {
    NS_TRY(check_batch(net, batch, x, y));
    NS_TRY(forward(net, x, batch));
    NS_CUDA(cudaMemcpyAsync(y, net->y, (size_t)batch * net->H * net->W * sizeof(float), cudaMemcpyDeviceToDevice,
                            net->stream));
    return NSSTAB_OK;
}

int unet_gradient(nsstab_unet* net, const float* x, const float* target, int batch, float* grad, double* loss) {
    NS_TRY(check_batch(net, batch, x, target));
    if (!grad || !loss) {
        set_error("unet_gradient: null argument");
        return NSSTAB_ERR_INVALID_ARG;
    }
    NS_TRY(forward(net, x, batch));
    NS_TRY(backward(net, target, batch, loss));
    NS_CUDA(cudaMemcpyAsync(grad, net->grad, net->count * sizeof(float), cudaMemcpyDeviceToDevice, net->stream));
    NS_CUDA(cudaStreamSynchronize(net->stream));
    return NSSTAB_OK;
}

int unet_train_step(nsstab_unet* net, const float* x, const float* target, int batch, float lr, float beta1,
                    float beta2, float eps, double* loss) {
    NS_TRY(check_batch(net, batch, x, target));
    if (!loss || !(lr > 0) || !(beta1 >= 0 && beta1 < 1) || !(beta2 >= 0 && beta2 < 1) || !(eps > 0)) {
        set_error("unet_train_step: need loss != NULL, lr > 0, 0 <= beta < 1, eps > 0");
        return NSSTAB_ERR_INVALID_ARG;
    }
    NS_TRY(forward(net, x, batch));
    NS_TRY(backward(net, target, batch, loss));
    net->step += 1;
    const float c1 = 1.f - std::pow(beta1, (float)net->step), c2 = 1.f - std::pow(beta2, (float)net->step);
    k_adam<<<grid_for(net->count, 256), 256, 0, net->stream>>>(net->theta, net->grad, net->m, net->v, net->wt, net->map,
                                                               net->count, lr, beta1, beta2, eps, c1, c2);
    NS_LAUNCH_CHECK();
    return NSSTAB_OK;
}

}  // extern "C"
