// Shared-memory Stockham FFT for the row and column passes of the stepper.
//
// A block transforms `nseq` complex sequences of length N = 2^logN (N >= 8)
// in place in shared memory.  Every thread owns 8 elements per pass:
// radix-8 passes while at least three factors of two remain, then one
// radix-4 (two butterflies per thread) or radix-2 (four butterflies per
// thread) pass.  The Stockham (self-sorting) index map is used, so input and
// output are both in natural order and no bit reversal is needed.
//
// Shared-memory layout: sequence f occupies S = padded_len(N) (or more)
// slots starting at s + f*S; element e sits at slot pad8(e) = e + e/8, which
// keeps the stride-8 stores of the first pass free of bank conflicts.
//
// Twiddles come from a precomputed table tw[e] = exp(-2 pi i e / Nt) of the
// longest transform length Nt of the grid (computed on the host in extended
// precision), read through the read-only cache: on GB300 the FP64 pipe is
// the scarce resource, so no sine or cosine is evaluated on the device.
#pragma once

#include "common.cuh"

namespace nsstab {

__host__ __device__ __forceinline__ int pad8(int i) { return i + (i >> 3); }
__host__ __device__ constexpr int padded_len(int n) { return n + (n >> 3); }

template <class T> struct Consts;
template <> struct Consts<double> { static constexpr double rsqrt2 = 0.70710678118654752440084436210485; };
template <> struct Consts<float> { static constexpr float rsqrt2 = 0.70710678118654752440f; };

// forward: X_k = sum_j x_j exp(-2 pi i jk/N); INV: exp(+2 pi i jk/N), unnormalised
template <bool INV, class C> __device__ __forceinline__ void dft4(C& a0, C& a1, C& a2, C& a3) {
    const C s02 = cadd(a0, a2), d02 = csub(a0, a2);
    const C s13 = cadd(a1, a3), d13 = csub(a1, a3);
    const C t = INV ? cmul_pi(d13) : cmul_mi(d13);
    a0 = cadd(s02, s13);
    a2 = csub(s02, s13);
    a1 = cadd(d02, t);
    a3 = csub(d02, t);
}

template <bool INV, class T> __device__ __forceinline__ void dft8(Cx<T>* v) {
    // decimation in frequency: X_{2k} = DFT4(a)_k, X_{2k+1} = DFT4(b)_k with
    // a_r = v_r + v_{r+4}, b_r = (v_r - v_{r+4}) W8^r, W8 = exp(-+ 2 pi i / 8)
    Cx<T> a0 = cadd(v[0], v[4]), b0 = csub(v[0], v[4]);
    Cx<T> a1 = cadd(v[1], v[5]), b1 = csub(v[1], v[5]);
    Cx<T> a2 = cadd(v[2], v[6]), b2 = csub(v[2], v[6]);
    Cx<T> a3 = cadd(v[3], v[7]), b3 = csub(v[3], v[7]);
    const T r = Consts<T>::rsqrt2;
    if (!INV) {
        b1 = mk<T>((b1.x + b1.y) * r, (b1.y - b1.x) * r);     // (1 - i)/sqrt2
        b2 = cmul_mi(b2);                                    // -i
        b3 = mk<T>((b3.y - b3.x) * r, -(b3.x + b3.y) * r);    // (-1 - i)/sqrt2
    } else {
        b1 = mk<T>((b1.x - b1.y) * r, (b1.x + b1.y) * r);     // (1 + i)/sqrt2
        b2 = cmul_pi(b2);                                    // +i
        b3 = mk<T>(-(b3.x + b3.y) * r, (b3.x - b3.y) * r);    // (-1 + i)/sqrt2
    }
    dft4<INV>(a0, a1, a2, a3);
    dft4<INV>(b0, b1, b2, b3);
    v[0] = a0; v[1] = b0; v[2] = a1; v[3] = b1;
    v[4] = a2; v[5] = b2; v[6] = a3; v[7] = b3;
}

template <bool INV, class T>
__device__ __forceinline__ Cx<T> twiddle(Cx<T> a, const Cx<T>* __restrict__ tw, int e) {
    const Cx<T> w = __ldg(tw + e);
    return INV ? cmulc(a, w) : cmul(a, w);
}

// In-place transform of nseq sequences (see file comment).  All threads of
// the block must call it.  Requirements: blockDim.x * 8 is a multiple of N;
// twshift = log2(Nt / N) for the table tw of length Nt.
template <bool INV, class T>
__device__ void fft_smem(Cx<T>* s, int logN, int S, int nseq, const Cx<T>* __restrict__ tw, int twshift) {
    using C = Cx<T>;
    const int t = threadIdx.x;
    const int lq = logN - 3;                    // log2(N/8): threads per sequence
    const int q = t & ((1 << lq) - 1);
    const int F = blockDim.x >> lq;             // sequences per round
    for (int f0 = 0; f0 < nseq; f0 += F) {
        const int f = f0 + (t >> lq);
        const bool act = f < nseq;
        C* d = s + (size_t)(act ? f : 0) * S;
        int nsl = 0;                            // log2 of the Stockham stride Ns
        int rem = logN;
        while (rem > 0) {
            C v[8];
            if (rem >= 3) {                     // ---- radix 8
                if (act) {
#pragma unroll
                    for (int r = 0; r < 8; ++r) v[r] = d[pad8(q + (r << lq))];
                }
                __syncthreads();
                if (act) {
                    const int k = q & ((1 << nsl) - 1);
                    if (nsl > 0) {
                        const int sh = logN - nsl - 3 + twshift;
#pragma unroll
                        for (int r = 1; r < 8; ++r) v[r] = twiddle<INV, T>(v[r], tw, (r * k) << sh);
                    }
                    dft8<INV, T>(v);
                    const int base = ((q - k) << 3) + k;
#pragma unroll
                    for (int r = 0; r < 8; ++r) d[pad8(base + (r << nsl))] = v[r];
                }
                __syncthreads();
                nsl += 3;
                rem -= 3;
            } else if (rem == 2) {              // ---- radix 4, two butterflies
                if (act) {
#pragma unroll
                    for (int u = 0; u < 2; ++u)
#pragma unroll
                        for (int r = 0; r < 4; ++r) v[4 * u + r] = d[pad8(q + (u << lq) + (r << (logN - 2)))];
                }
                __syncthreads();
                if (act) {
#pragma unroll
                    for (int u = 0; u < 2; ++u) {
                        const int b = q + (u << lq);
                        const int k = b & ((1 << nsl) - 1);
                        if (nsl > 0) {
                            const int sh = logN - nsl - 2 + twshift;
#pragma unroll
                            for (int r = 1; r < 4; ++r) v[4 * u + r] = twiddle<INV, T>(v[4 * u + r], tw, (r * k) << sh);
                        }
                        dft4<INV>(v[4 * u], v[4 * u + 1], v[4 * u + 2], v[4 * u + 3]);
                        const int base = ((b - k) << 2) + k;
#pragma unroll
                        for (int r = 0; r < 4; ++r) d[pad8(base + (r << nsl))] = v[4 * u + r];
                    }
                }
                __syncthreads();
                nsl += 2;
                rem = 0;
            } else {                            // ---- radix 2, four butterflies
                if (act) {
#pragma unroll
                    for (int u = 0; u < 4; ++u) {
                        v[2 * u] = d[pad8(q + (u << lq))];
                        v[2 * u + 1] = d[pad8(q + (u << lq) + (1 << (logN - 1)))];
                    }
                }
                __syncthreads();
                if (act) {
#pragma unroll
                    for (int u = 0; u < 4; ++u) {
                        const int b = q + (u << lq);
                        const int k = b & ((1 << nsl) - 1);
                        if (nsl > 0) v[2 * u + 1] = twiddle<INV, T>(v[2 * u + 1], tw, k << (logN - nsl - 1 + twshift));
                        const C x0 = v[2 * u], x1 = v[2 * u + 1];
                        const int base = ((b - k) << 1) + k;
                        d[pad8(base)] = cadd(x0, x1);
                        d[pad8(base + (1 << nsl))] = csub(x0, x1);
                    }
                }
                __syncthreads();
                nsl += 1;
                rem = 0;
            }
        }
    }
}

}  // namespace nsstab
