// Shared-memory Stockham FFT for the row and column passes of the stepper.
//
// A block transforms `nseq` complex sequences of length N = 2^logN in place
// in shared memory.  Every thread owns E = 2, 4 or 8 elements per pass
// (template parameter): radix-E passes while enough factors of two remain,
// then one smaller-radix pass with several butterflies per thread.  Fewer
// elements per thread means more warps for the same transform, which is
// what small grids need to occupy all four SM sub-partitions (on GB300 a
// warp-wide FP64 instruction holds a sub-partition's FP64 unit for 64
// cycles, so each sub-partition needs its own warp).  The Stockham (self-sorting) index map is used, so input and
// output are both in natural order and no bit reversal is needed.
//
// Shared-memory layout: sequence f occupies S = seq_stride(...) >= N (FP32:
// N + N/16) slots starting at s + f*S; element e sits at slot sw<T>(e),
// which keeps the strided stores of the early passes free of bank
// conflicts: FP64 and double-float XOR-swizzle within each 128-byte bank
// row; FP32 inserts one pad slot after every 16 elements, so that slot(e +
// 16 j) = slot(e) + 17 j and the reads of a pass (stride N/R) and the writes
// of the passes with stride >= 16 are linear in r: one address per pass
// instead of one per element.
//
// Twiddles come from precomputed per-pass tables (twiddle_table_len; built
// on the host in extended precision) read through the read-only cache: on
// GB300 the FP64 pipe is the scarce resource, so no sine or cosine is
// evaluated on the device, and each butterfly's twiddles are one contiguous
// row so that the loads of a warp are coalesced.
//
// FP32 transforms carry every twiddle as hi + lo (lo = the FP32 rounding
// error of hi) and fold the lo product into the fused multiply-adds before
// their final rounding; the radix-8 constant 1/sqrt(2) is split the same
// way.  A twiddle rounded to FP32 makes the transform a fixed, slightly
// wrong linear map, and a time-stepper applies that same map at every step,
// so its error adds up linearly over a run (about 1e-5 relative after a few
// hundred steps, which then bounds the accuracy of the eigenvalues); with
// the split only the data-dependent rounding of the arithmetic remains.
#pragma once

#include <type_traits>

#include "common.cuh"

namespace nsstab {

// Shared-memory slot of element i of a sequence: an XOR swizzle inside each
// 128-byte bank row (16 float2 or 8 double2 elements) that keeps both the
// unit-stride accesses and the stride-8 stores of the first radix-8 pass
// free of bank conflicts, without padding.
template <class T> __device__ __forceinline__ int sw(int i);
template <> __device__ __forceinline__ int sw<float>(int i) { return i + (i >> 4); }
template <> __device__ __forceinline__ int sw<double>(int i) { return i ^ ((i >> 3) & 7); }
template <> __device__ __forceinline__ int sw<df64>(int i) { return i ^ ((i >> 3) & 7); }
// Slots a sequence of n elements occupies (elem_words = element size / 4
// bytes; 2 is FP32 complex, whose layout pads one slot per 16 elements).
__host__ __device__ constexpr int padded_len(int n, int elem_words) { return elem_words == 2 ? n + (n >> 4) : n; }
// Distance (in elements) between consecutive sequences in shared memory.
// When `rp` sequences share one shared-memory wavefront (element-interleaved
// staging loops, or short sequences several to a warp), their starts are
// spread over the 32 four-byte banks, 32/rp banks apart.
__host__ __device__ inline int seq_stride(int n, int rp, int elem_words) {
    int s = padded_len(n, elem_words);
    if (rp <= 1) return s;
    const int target = (32 / rp) & 31;
    for (int i = 0; i < 32; ++i, ++s)
        if (((s * elem_words) & 31) == target) return s;
    return padded_len(n, elem_words) + 1;
}

// Twiddle tables, one per elements-per-thread choice LE: for every pass
// with Stockham stride Ns and radix R (in the order fft_smem runs them), R
// rows of Ns entries exp(-2 pi i r k / (Ns R)), r < R, k < Ns.  Consecutive
// threads of a pass have consecutive k, so the loads of a warp for one r
// are contiguous.  Length < 2N entries (each kTwWidth<T> Cx<T> slots).
inline int twiddle_table_len(int logN, int LE) {
    int len = 0, nsl = 0, rem = logN;
    while (rem >= LE) {
        len += (1 << nsl) << LE;
        nsl += LE;
        rem -= LE;
    }
    if (rem > 0) len += (1 << nsl) << rem;
    return len;
}

// Cx<T> slots per twiddle entry: FP32 tables store hi and lo side by side.
template <class T> constexpr int kTwWidth = std::is_same<T, float>::value ? 2 : 1;

template <class T> struct Consts;
template <> struct Consts<double> { static constexpr double rsqrt2 = 0.70710678118654752440084436210485; };
template <> struct Consts<float> {
    static constexpr float rsqrt2 = 0.70710678118654752440f;
    static constexpr float rsqrt2_lo = 1.21016175e-08f;   // 1/sqrt(2) - rsqrt2
};
template <> struct Consts<df64> { static constexpr df64 rsqrt2 = df64(0.70710677f, 1.21016175e-08f); };

// s / sqrt(2), with the FP32 constant's rounding error compensated
template <class T> __device__ __forceinline__ T mul_rsqrt2(T s) {
    if constexpr (std::is_same<T, float>::value) {
        return __fmaf_rn(s, Consts<float>::rsqrt2, s * Consts<float>::rsqrt2_lo);
    } else {
        return s * Consts<T>::rsqrt2;
    }
}

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
    if (!INV) {
        b1 = mk<T>(mul_rsqrt2<T>(b1.x + b1.y), mul_rsqrt2<T>(b1.y - b1.x));     // (1 - i)/sqrt2
        b2 = cmul_mi(b2);                                                      // -i
        b3 = mk<T>(mul_rsqrt2<T>(b3.y - b3.x), -mul_rsqrt2<T>(b3.x + b3.y));    // (-1 - i)/sqrt2
    } else {
        b1 = mk<T>(mul_rsqrt2<T>(b1.x - b1.y), mul_rsqrt2<T>(b1.x + b1.y));     // (1 + i)/sqrt2
        b2 = cmul_pi(b2);                                                      // +i
        b3 = mk<T>(-mul_rsqrt2<T>(b3.x + b3.y), mul_rsqrt2<T>(b3.x - b3.y));    // (-1 + i)/sqrt2
    }
    dft4<INV>(a0, a1, a2, a3);
    dft4<INV>(b0, b1, b2, b3);
    v[0] = a0; v[1] = b0; v[2] = a1; v[3] = b1;
    v[4] = a2; v[5] = b2; v[6] = a3; v[7] = b3;
}

// a * w_e (INV: a * conj(w_e)) for twiddle entry e of table tw
template <bool INV, class T>
__device__ __forceinline__ Cx<T> twiddle(Cx<T> a, const Cx<T>* __restrict__ tw, int e) {
    if constexpr (std::is_same<T, float>::value) {
        const float4 q = __ldg(reinterpret_cast<const float4*>(tw) + e);   // hi (x, y), lo (z, w)
        float re, im;
        if (!INV) {
            const float lr = a.x * q.z - a.y * q.w, li = a.x * q.w + a.y * q.z;
            re = __fmaf_rn(a.x, q.x, __fmaf_rn(-a.y, q.y, lr));
            im = __fmaf_rn(a.x, q.y, __fmaf_rn(a.y, q.x, li));
        } else {
            const float lr = a.x * q.z + a.y * q.w, li = a.y * q.z - a.x * q.w;
            re = __fmaf_rn(a.x, q.x, __fmaf_rn(a.y, q.y, lr));
            im = __fmaf_rn(a.y, q.x, __fmaf_rn(-a.x, q.y, li));
        }
        return mk<float>(re, im);
    } else {
        const Cx<T> w = ldg_c(tw + e);
        return INV ? cmulc(a, w) : cmul(a, w);
    }
}

template <bool INV, class T, int LR> __device__ __forceinline__ void dft_r(Cx<T>* v) {
    if (LR == 3) {
        dft8<INV, T>(v);
    } else if (LR == 2) {
        dft4<INV>(v[0], v[1], v[2], v[3]);
    } else {
        const Cx<T> a = v[0], b = v[1];
        v[0] = cadd(a, b);
        v[1] = csub(a, b);
    }
}

// One Stockham pass of radix R = 2^LR for a thread owning E = 2^LE elements
// (E/R butterflies).  Butterfly b reads b + r N/R and writes
// (b - k) R + k + r Ns with k = b mod Ns, after twiddling input r by
// W_N^(r k N/(Ns R)).
template <bool INV, class T, int LE, int LR>
__device__ __forceinline__ void stockham_pass(Cx<T>* d, int q, int lq, int logN, int nsl,
                                              const Cx<T>* __restrict__ tw, bool act) {
    constexpr int E = 1 << LE, R = 1 << LR, U = E / R;
    constexpr bool PAD = std::is_same<T, float>::value;   // sw<float>: linear in steps of 16
    Cx<T> v[E];
    if (act) {
        const int M = 1 << (logN - LR);   // read stride
        if (PAD && M >= 16) {
            const int Mp = M + (M >> 4);
#pragma unroll
            for (int u = 0; u < U; ++u) {
                const Cx<T>* p = d + sw<T>(q + (u << lq));
#pragma unroll
                for (int r = 0; r < R; ++r) v[u * R + r] = p[r * Mp];
            }
        } else {
#pragma unroll
            for (int u = 0; u < U; ++u)
#pragma unroll
                for (int r = 0; r < R; ++r) v[u * R + r] = d[sw<T>(q + (u << lq) + (r << (logN - LR)))];
        }
    }
    __syncthreads();
    if (act) {
        const int Ns = 1 << nsl;
#pragma unroll
        for (int u = 0; u < U; ++u) {
            const int b = q + (u << lq);
            const int k = b & (Ns - 1);
            if (nsl > 0) {
                const Cx<T>* twk = tw + kTwWidth<T> * k;
#pragma unroll
                for (int r = 1; r < R; ++r) v[u * R + r] = twiddle<INV, T>(v[u * R + r], twk, r * Ns);
            }
            dft_r<INV, T, LR>(v + u * R);
            const int base = ((b - k) << LR) + k;
            if (PAD && Ns >= 16) {
                Cx<T>* p = d + sw<T>(base);
                const int Np = Ns + (Ns >> 4);
#pragma unroll
                for (int r = 0; r < R; ++r) p[r * Np] = v[u * R + r];
            } else {
#pragma unroll
                for (int r = 0; r < R; ++r) d[sw<T>(base + r * Ns)] = v[u * R + r];
            }
        }
    }
    __syncthreads();
}

// In-place transform of nseq sequences, sequence f at seq(f) (a device
// functor returning its shared-memory start).  All threads of the block must
// call it.  Every thread owns E = 2^LE elements per pass: radix-E passes,
// then one smaller radix for the remaining factors.  Requirements: logN >=
// LE; blockDim.x >= N/E; tw is the twiddle table of this N and LE
// (twiddle_table_len entries).
template <bool INV, class T, int LE, class SeqPtr>
__device__ void fft_smem_seqs(SeqPtr seq, int logN, int nseq, const Cx<T>* __restrict__ tw) {
    const int t = threadIdx.x;
    const int lq = logN - LE;                   // log2(N/E): threads per sequence
    const int q = t & ((1 << lq) - 1);
    const int F = blockDim.x >> lq;             // sequences per round
    for (int f0 = 0; f0 < nseq; f0 += F) {
        const int f = f0 + (t >> lq);
        const bool act = f < nseq;
        Cx<T>* d = seq(act ? f : 0);
        int nsl = 0;
        int rem = logN;
        const Cx<T>* twp = tw;   // start of this pass's rows
        while (rem >= LE) {
            stockham_pass<INV, T, LE, LE>(d, q, lq, logN, nsl, twp, act);
            twp += kTwWidth<T> * ((1 << nsl) << LE);
            nsl += LE;
            rem -= LE;
        }
        if (LE == 3 && rem == 2) stockham_pass<INV, T, LE, (LE == 3 ? 2 : 1)>(d, q, lq, logN, nsl, twp, act);
        if (rem == 1) stockham_pass<INV, T, LE, 1>(d, q, lq, logN, nsl, twp, act);
    }
}

// In-place transform of nseq sequences stored S elements apart from s (see
// the file comment and fft_smem_seqs).  blockDim.x * E is a multiple of N.
template <bool INV, class T, int LE>
__device__ void fft_smem(Cx<T>* s, int logN, int S, int nseq, const Cx<T>* __restrict__ tw) {
    fft_smem_seqs<INV, T, LE>([=](int f) { return s + (size_t)f * S; }, logN, nseq, tw);
}

}  // namespace nsstab
