// FP64 tall-skinny kernels of the Krylov layer: the classical Gram-Schmidt
// products of Algorithm 1 (h = V^T w, w -= V h, applied twice = CGS2), norms
// and the basis contraction V Q of the Krylov-Schur truncation / Ritz vector
// assembly (Sec. 3.2.2).  The basis V is column-major: column k of length n
// starts at V + k*ldv.  Reductions use a fixed grid and a fixed summation
// order, so results are bit-reproducible run to run.
#include <algorithm>
#include <vector>

#include "stepper.cuh"

namespace nsstab {

static const int kGsBlocks = 304;   // two blocks per SM on a 152-SM GB300
static const int kGsThreads = 256;
static const int kColGroup = 8;     // columns accumulated per pass over w

// partial[b * ldp + c] = sum over block b's row range of V[c][i] * w[i], c < j
__global__ void k_gs_dot(const double* __restrict__ V, long ldv, long n, int j,
                         const double* __restrict__ w, double* __restrict__ partial, int ldp) {
    const long chunk = (n + gridDim.x - 1) / gridDim.x;
    const long r0 = (long)blockIdx.x * chunk;
    const long r1 = min(n, r0 + chunk);
    __shared__ double red[kColGroup][kGsThreads / 32];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    for (int c0 = 0; c0 < j; c0 += kColGroup) {
        const int nc = min(kColGroup, j - c0);
        double acc[kColGroup];
#pragma unroll
        for (int cc = 0; cc < kColGroup; ++cc) acc[cc] = 0.0;
        for (long i = r0 + threadIdx.x; i < r1; i += blockDim.x) {
            const double wi = w[i];
#pragma unroll
            for (int cc = 0; cc < kColGroup; ++cc)
                if (cc < nc) acc[cc] = fma(V[(long)(c0 + cc) * ldv + i], wi, acc[cc]);
        }
#pragma unroll
        for (int cc = 0; cc < kColGroup; ++cc) {
            double a = acc[cc];
            for (int o = 16; o > 0; o >>= 1) a += __shfl_down_sync(0xffffffffu, a, o);
            if (lane == 0) red[cc][warp] = a;
        }
        __syncthreads();
        if (threadIdx.x < nc) {
            double s = 0.0;
            for (int wv = 0; wv < (int)(blockDim.x >> 5); ++wv) s += red[threadIdx.x][wv];
            partial[(long)blockIdx.x * ldp + c0 + threadIdx.x] = s;
        }
        __syncthreads();
    }
}

// out[c] = sum_b partial[b * ldp + c]  (fixed order over b)
__global__ void k_gs_reduce(const double* __restrict__ partial, int nb, int ldp, int j, double* __restrict__ out) {
    for (int c = threadIdx.x; c < j; c += blockDim.x) {
        double s = 0.0;
        for (int b = 0; b < nb; ++b) s += partial[(long)b * ldp + c];
        out[c] = s;
    }
}

// out[c] = sum_b partial[b * ldp + c] for c < j, over many blocks: each block
// takes 32 columns, its 8 warps sum interleaved rows of partials, and warp 0
// adds the 8 warp sums in a fixed order (bit-reproducible run to run).
// member blockIdx.y: partial + member * nb * ldp, out + member * ldo; js
// (optional) gives a per-member column count (<= 0: member skipped).
__global__ void k_gs_reduce_par(const double* __restrict__ partial, int nb, int ldp, int j,
                                const int* __restrict__ js, double* __restrict__ out, int ldo) {
    const int b = blockIdx.y;
    if (js) j = js[b];
    const int lane = threadIdx.x & 31, wv = threadIdx.x >> 5, nw = blockDim.x >> 5;
    const int c = blockIdx.x * 32 + lane;
    if (j <= 0 || blockIdx.x * 32 >= j) return;
    partial += (size_t)b * nb * ldp;
    __shared__ double red[32][33];
    double s = 0.0;
    if (c < j)
        for (int r = wv; r < nb; r += nw) s += partial[(long)r * ldp + c];
    red[wv][lane] = s;
    __syncthreads();
    if (wv == 0 && c < j) {
        double t = 0.0;
        for (int w = 0; w < nw; ++w) t += red[w][lane];
        out[(size_t)b * ldo + c] = t;
    }
}

// w[i] -= sum_c V[c][i] h[c]
__global__ void k_gs_update(double* __restrict__ w, const double* __restrict__ V, long ldv, long n, int j,
                            const double* __restrict__ h) {
    extern __shared__ double hs[];
    for (int c = threadIdx.x; c < j; c += blockDim.x) hs[c] = h[c];
    __syncthreads();
    for (long i = (long)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (long)gridDim.x * blockDim.x) {
        double acc = 0.0;
        for (int c = 0; c < j; ++c) acc = fma(V[(long)c * ldv + i], hs[c], acc);
        w[i] -= acc;
    }
}

// dst = a x + b y (dst may alias x or y)
__global__ void k_axpby(double* dst, double a, const double* x, double b, const double* y, long n) {
    for (long i = (long)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (long)gridDim.x * blockDim.x)
        dst[i] = a * x[i] + b * y[i];
}

__global__ void k_scale(double* __restrict__ dst, const double* __restrict__ src, long n, double s) {
    for (long i = (long)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (long)gridDim.x * blockDim.x)
        dst[i] = src[i] * s;
}

// out[c][i] = sum_k V[k][i] C[c*ldc + k], c < p  (out must not alias V)
__global__ void k_combine(const double* __restrict__ V, long ldv, long n, int m, const double* __restrict__ C,
                          int ldc, int p, double* __restrict__ out, long ldo) {
    const int G = 8;
    for (long i = (long)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (long)gridDim.x * blockDim.x) {
        for (int c0 = 0; c0 < p; c0 += G) {
            double acc[G];
#pragma unroll
            for (int g = 0; g < G; ++g) acc[g] = 0.0;
            for (int k = 0; k < m; ++k) {
                const double v = V[(long)k * ldv + i];
#pragma unroll
                for (int g = 0; g < G; ++g)
                    if (c0 + g < p) acc[g] = fma(v, __ldg(C + (long)(c0 + g) * ldc + k), acc[g]);
            }
#pragma unroll
            for (int g = 0; g < G; ++g)
                if (c0 + g < p) out[(long)(c0 + g) * ldo + i] = acc[g];
        }
    }
}

// ----------------------------------------------------- batched variants
// Member b (blockIdx.y) works on its own basis V[b] (column-major, leading
// dimension ldv), vector w[b] and column count j[b]; j[b] <= 0 leaves w[b]
// alone in the products (the norm pass uses its own count array).

__global__ void k_gs_dot_b(const double* const* __restrict__ Vs, long ldv, long n, const int* __restrict__ js,
                           const double* const* __restrict__ ws, double* __restrict__ partial, int ldp,
                           const long* __restrict__ ns) {
    const int b = blockIdx.y;
    const int j = js[b];
    if (j <= 0) return;
    if (ns) ldv = n = ns[b];   // members of different lengths: ldv = n per member
    const double* V = Vs[b];
    const double* w = ws[b];
    double* part = partial + (size_t)b * gridDim.x * ldp;
    const long chunk = (n + gridDim.x - 1) / gridDim.x;
    const long r0 = (long)blockIdx.x * chunk;
    const long r1 = min(n, r0 + chunk);
    __shared__ double red[kColGroup][kGsThreads / 32];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    for (int c0 = 0; c0 < j; c0 += kColGroup) {
        const int nc = min(kColGroup, j - c0);
        double acc[kColGroup];
#pragma unroll
        for (int cc = 0; cc < kColGroup; ++cc) acc[cc] = 0.0;
        for (long i = r0 + threadIdx.x; i < r1; i += blockDim.x) {
            const double wi = w[i];
#pragma unroll
            for (int cc = 0; cc < kColGroup; ++cc)
                if (cc < nc) acc[cc] = fma(V[(long)(c0 + cc) * ldv + i], wi, acc[cc]);
        }
#pragma unroll
        for (int cc = 0; cc < kColGroup; ++cc) {
            double a = acc[cc];
            for (int o = 16; o > 0; o >>= 1) a += __shfl_down_sync(0xffffffffu, a, o);
            if (lane == 0) red[cc][warp] = a;
        }
        __syncthreads();
        if (threadIdx.x < nc) {
            double s = 0.0;
            for (int wv = 0; wv < (int)(blockDim.x >> 5); ++wv) s += red[threadIdx.x][wv];
            part[(long)blockIdx.x * ldp + c0 + threadIdx.x] = s;
        }
        __syncthreads();
    }
}

__global__ void k_gs_update_b(double* const* __restrict__ ws, const double* const* __restrict__ Vs, long ldv, long n,
                              const int* __restrict__ js, const double* __restrict__ h, int ldp,
                              const long* __restrict__ ns) {
    const int b = blockIdx.y;
    const int j = js[b];
    if (j <= 0) return;
    if (ns) ldv = n = ns[b];
    extern __shared__ double hs[];
    for (int c = threadIdx.x; c < j; c += blockDim.x) hs[c] = h[(size_t)b * ldp + c];
    __syncthreads();
    double* w = ws[b];
    const double* V = Vs[b];
    for (long i = (long)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (long)gridDim.x * blockDim.x) {
        double acc = 0.0;
        for (int c = 0; c < j; ++c) acc = fma(V[(long)c * ldv + i], hs[c], acc);
        w[i] -= acc;
    }
}

__global__ void k_scale_b(double* const* __restrict__ ws, long n, const double* __restrict__ s,
                          const long* __restrict__ ns) {
    double* w = ws[blockIdx.y];
    if (!w) return;
    if (ns) n = ns[blockIdx.y];
    const double f = s[blockIdx.y];
    for (long i = (long)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (long)gridDim.x * blockDim.x) w[i] *= f;
}

// ------------------------------------------------ blocked Gram-Schmidt
// Block form of the Gram-Schmidt step for block Krylov methods: the b new
// columns W of a set are projected against its first J orthonormal basis
// columns in one tall-skinny product pair, H = V_J^T W (J x b) and
// W -= V_J H, so V is read once per pass for all b columns instead of once
// per column.  Set s = blockIdx.z (dot) / blockIdx.y (update); J[s] <= 0
// skips the set.  W's columns are ldw apart; H is stored [c * b + q].

static const int kBgsCols = 4;   // basis columns per block row of the dot product

// partial[s][blk][c * B + q] = sum over block blk's row range of V[c][i] W[q][i],
// for the kBgsCols columns c of block row blockIdx.y
template <int B>
__global__ void __launch_bounds__(256) k_bgs_dot(const double* const* __restrict__ Vs, long ldv, long n,
                                                 const int* __restrict__ Js, const double* const* __restrict__ Ws,
                                                 long ldw, double* __restrict__ partial, int ldp) {
    const int s = blockIdx.z;
    const int J = Js[s];
    const int c0 = blockIdx.y * kBgsCols;
    if (J <= 0 || c0 >= J) return;
    const double* V = Vs[s];
    const double* W = Ws[s];
    const long chunk = (n + gridDim.x - 1) / gridDim.x;
    const long r0 = (long)blockIdx.x * chunk;
    const long r1 = min(n, r0 + chunk);
    const int nc = min(kBgsCols, J - c0);
    double acc[kBgsCols][B];
#pragma unroll
    for (int cc = 0; cc < kBgsCols; ++cc)
#pragma unroll
        for (int q = 0; q < B; ++q) acc[cc][q] = 0.0;
    for (long i = r0 + threadIdx.x; i < r1; i += blockDim.x) {
        double w[B];
#pragma unroll
        for (int q = 0; q < B; ++q) w[q] = W[(long)q * ldw + i];
#pragma unroll
        for (int cc = 0; cc < kBgsCols; ++cc) {
            if (cc < nc) {
                const double v = V[(long)(c0 + cc) * ldv + i];
#pragma unroll
                for (int q = 0; q < B; ++q) acc[cc][q] = fma(v, w[q], acc[cc][q]);
            }
        }
    }
    __shared__ double red[kBgsCols * B][8];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
#pragma unroll
    for (int cc = 0; cc < kBgsCols; ++cc)
#pragma unroll
        for (int q = 0; q < B; ++q) {
            double a = acc[cc][q];
            for (int o = 16; o > 0; o >>= 1) a += __shfl_down_sync(0xffffffffu, a, o);
            if (lane == 0) red[cc * B + q][warp] = a;
        }
    __syncthreads();
    const int t = threadIdx.x;
    if (t < nc * B) {
        double sum = 0.0;
        for (int wv = 0; wv < (int)(blockDim.x >> 5); ++wv) sum += red[t][wv];
        partial[((size_t)s * gridDim.x + blockIdx.x) * ldp + (size_t)c0 * B + t] = sum;
    }
}

// W[q][i] -= sum_c V[c][i] H[c * B + q]
template <int B>
__global__ void __launch_bounds__(256) k_bgs_update(double* const* __restrict__ Ws, long ldw,
                                                    const double* const* __restrict__ Vs, long ldv, long n,
                                                    const int* __restrict__ Js, const double* __restrict__ H,
                                                    int ldh) {
    const int s = blockIdx.y;
    const int J = Js[s];
    if (J <= 0) return;
    extern __shared__ double hs[];
    for (int e = threadIdx.x; e < J * B; e += blockDim.x) hs[e] = H[(size_t)s * ldh + e];
    __syncthreads();
    double* W = Ws[s];
    const double* V = Vs[s];
    for (long i = (long)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (long)gridDim.x * blockDim.x) {
        double acc[B];
#pragma unroll
        for (int q = 0; q < B; ++q) acc[q] = 0.0;
        for (int c = 0; c < J; ++c) {
            const double v = V[(long)c * ldv + i];
#pragma unroll
            for (int q = 0; q < B; ++q) acc[q] = fma(v, hs[c * B + q], acc[q]);
        }
#pragma unroll
        for (int q = 0; q < B; ++q) W[(long)q * ldw + i] -= acc[q];
    }
}

template <int B>
static int bgs_pass(int S, const double* const* Vd, long ldv, long n, const int* Jd, int Jmax, double* const* Wd,
                    long ldw, double* partial, int nbx, int ldp, double* Hout, cudaStream_t stream) {
    const dim3 gd(nbx, (Jmax + kBgsCols - 1) / kBgsCols, S);
    k_bgs_dot<B><<<gd, 256, 0, stream>>>(Vd, ldv, n, Jd, (const double* const*)Wd, ldw, partial, ldp);
    k_gs_reduce_par<<<dim3((Jmax * B + 31) / 32, S), 256, 0, stream>>>(partial, nbx, ldp, Jmax * B, nullptr, Hout,
                                                                        ldp);
    const int ub = std::max(16, 4 * 152 / S);
    k_bgs_update<B><<<dim3(ub, S), 256, (size_t)Jmax * B * sizeof(double), stream>>>(Wd, ldw, Vd, ldv, n, Jd,
                                                                                      Hout, ldp);
    NS_LAUNCH_CHECK();
    return NSSTAB_OK;
}

int bcgs2_batch(int S, const double* const* V, long ldv, long n, const int* J, double* const* W, long ldw, int b,
                double* H, int ldh, GsBatch& ws, cudaStream_t stream) {
    if (b < 1 || b > kMaxGsBlock) {
        set_error("block Gram-Schmidt: block size out of range");
        return NSSTAB_ERR_INVALID_ARG;
    }
    int Jmax = 0;
    for (int s = 0; s < S; ++s) Jmax = std::max(Jmax, J[s]);
    if (Jmax <= 0) return NSSTAB_OK;
    const int ldp = Jmax * b;
    NS_TRY(ws.alloc(S, ldp));
    std::vector<int> jh(S);
    std::vector<const double*> ph(2 * (size_t)S);
    for (int s = 0; s < S; ++s) {
        jh[s] = J[s];
        ph[s] = V[s];
        ph[S + s] = W[s];
    }
    NS_CUDA(cudaMemcpyAsync(ws.jdev, jh.data(), S * sizeof(int), cudaMemcpyHostToDevice, stream));
    NS_CUDA(cudaMemcpyAsync(ws.ptrs, ph.data(), ph.size() * sizeof(double*), cudaMemcpyHostToDevice, stream));
    const double* const* Vd = (const double* const*)ws.ptrs;
    double* const* Wd = ws.ptrs + S;
    // partial sums [S][nbx][ldp] fit the workspace's [S][grid][max_cols]
    const int rows_of_blocks = (Jmax + kBgsCols - 1) / kBgsCols;
    const int nbx = std::max(8, std::min(ws.grid, 4 * 152 / std::max(1, rows_of_blocks * S)));
    double* h1 = ws.hdev;
    double* h2 = ws.hdev + (size_t)S * ldp;
#define NS_BGS(BB)                                                                                          \
    do {                                                                                                    \
        NS_TRY(bgs_pass<BB>(S, Vd, ldv, n, ws.jdev, Jmax, Wd, ldw, ws.partial, nbx, ldp, h1, stream));      \
        NS_TRY(bgs_pass<BB>(S, Vd, ldv, n, ws.jdev, Jmax, Wd, ldw, ws.partial, nbx, ldp, h2, stream));      \
    } while (0)
    switch (b) {
        case 1: NS_BGS(1); break;
        case 2: NS_BGS(2); break;
        case 3: NS_BGS(3); break;
        case 4: NS_BGS(4); break;
        case 5: NS_BGS(5); break;
        case 6: NS_BGS(6); break;
        case 7: NS_BGS(7); break;
        default: NS_BGS(8); break;
    }
#undef NS_BGS
    NS_CUDA(cudaMemcpyAsync(ws.hhost, ws.hdev, (size_t)2 * S * ldp * sizeof(double), cudaMemcpyDeviceToHost,
                            stream));
    NS_CUDA(cudaStreamSynchronize(stream));
    for (int s = 0; s < S; ++s)
        for (int e = 0; e < J[s] * b; ++e)
            H[(size_t)s * ldh + e] = ws.hhost[(size_t)s * ldp + e] + ws.hhost[(size_t)(S + s) * ldp + e];
    return NSSTAB_OK;
}

int GsBatch::alloc(int nmem, int cols) {
    if (nmem <= B && cols <= max_cols) return NSSTAB_OK;
    release();
    B = nmem;
    max_cols = cols;
    grid = 152;
    const size_t ph = (size_t)B * 3 * max_cols;
    NS_CUDA(cudaMalloc(&partial, (size_t)B * grid * max_cols * sizeof(double)));
    NS_CUDA(cudaMalloc(&hdev, ph * sizeof(double)));
    NS_CUDA(cudaMalloc(&jdev, (size_t)B * 2 * sizeof(int)));
    NS_CUDA(cudaMalloc(&ptrs, (size_t)B * 2 * sizeof(double*)));
    NS_CUDA(cudaMalloc(&sdev, (size_t)B * sizeof(double)));
    NS_CUDA(cudaMalloc(&ndev, (size_t)B * sizeof(long)));
    NS_CUDA(cudaMallocHost(&hhost, ph * sizeof(double)));
    return NSSTAB_OK;
}

void GsBatch::release() {
    if (partial) cudaFree(partial);
    if (hdev) cudaFree(hdev);
    if (jdev) cudaFree(jdev);
    if (ptrs) cudaFree(ptrs);
    if (sdev) cudaFree(sdev);
    if (ndev) cudaFree(ndev);
    if (hhost) cudaFreeHost(hhost);
    partial = hdev = sdev = hhost = nullptr;
    ndev = nullptr;
    jdev = nullptr;
    ptrs = nullptr;
    B = max_cols = 0;
}

// CGS2 of w[b] against the first j[b] columns of V[b] for every member with
// j[b] >= 0 (j[b] = 0: norm only; j[b] < 0: member skipped); h[b][0..j[b])
// and beta[b] = ||w[b]|| to the host.  One synchronisation.
int cgs2_batch(int nmem, const double* const* V, long ldv, long n, const int* j, double* const* w,
               double* h /*host [nmem][ldh]*/, int ldh, double* beta, GsBatch& ws, cudaStream_t stream,
               const long* nm) {
    int jmax = 1;
    for (int b = 0; b < nmem; ++b) jmax = std::max(jmax, j[b]);
    NS_TRY(ws.alloc(nmem, jmax));
    const long* nd = nullptr;
    if (nm) {
        NS_CUDA(cudaMemcpyAsync(ws.ndev, nm, nmem * sizeof(long), cudaMemcpyHostToDevice, stream));
        nd = ws.ndev;
    }
    const int ldp = ws.max_cols;
    std::vector<int> jh(2 * (size_t)nmem);
    std::vector<const double*> ph(2 * (size_t)nmem);
    for (int b = 0; b < nmem; ++b) {
        jh[b] = j[b];
        jh[nmem + b] = j[b] >= 0 ? 1 : 0;   // j < 0: member inactive in this call
        ph[b] = V[b];
        ph[nmem + b] = w[b];
    }
    NS_CUDA(cudaMemcpyAsync(ws.jdev, jh.data(), jh.size() * sizeof(int), cudaMemcpyHostToDevice, stream));
    NS_CUDA(cudaMemcpyAsync(ws.ptrs, ph.data(), ph.size() * sizeof(double*), cudaMemcpyHostToDevice, stream));
    const double* const* Vd = (const double* const*)ws.ptrs;
    double* const* wd = ws.ptrs + nmem;
    const int* jd = ws.jdev;
    const int* one = ws.jdev + nmem;
    double* h1 = ws.hdev;
    double* h2 = ws.hdev + (size_t)nmem * ldp;
    double* b2 = ws.hdev + 2 * (size_t)nmem * ldp;   // [nmem] spaced by ldp
    const dim3 g(ws.grid, nmem);
    const size_t sm = (size_t)jmax * sizeof(double);
    const dim3 gr((jmax + 31) / 32, nmem);
    k_gs_dot_b<<<g, kGsThreads, 0, stream>>>(Vd, ldv, n, jd, (const double* const*)wd, ws.partial, ldp, nd);
    k_gs_reduce_par<<<gr, 256, 0, stream>>>(ws.partial, ws.grid, ldp, 0, jd, h1, ldp);
    k_gs_update_b<<<dim3(2 * ws.grid, nmem), kGsThreads, sm, stream>>>(wd, Vd, ldv, n, jd, h1, ldp, nd);
    k_gs_dot_b<<<g, kGsThreads, 0, stream>>>(Vd, ldv, n, jd, (const double* const*)wd, ws.partial, ldp, nd);
    k_gs_reduce_par<<<gr, 256, 0, stream>>>(ws.partial, ws.grid, ldp, 0, jd, h2, ldp);
    k_gs_update_b<<<dim3(2 * ws.grid, nmem), kGsThreads, sm, stream>>>(wd, Vd, ldv, n, jd, h2, ldp, nd);
    k_gs_dot_b<<<g, kGsThreads, 0, stream>>>((const double* const*)wd, n, n, one, (const double* const*)wd,
                                             ws.partial, ldp, nd);
    k_gs_reduce_par<<<dim3(1, nmem), 256, 0, stream>>>(ws.partial, ws.grid, ldp, 0, one, b2, ldp);
    NS_LAUNCH_CHECK();
    NS_CUDA(cudaMemcpyAsync(ws.hhost, ws.hdev, (size_t)3 * nmem * ldp * sizeof(double), cudaMemcpyDeviceToHost,
                            stream));
    NS_CUDA(cudaStreamSynchronize(stream));
    for (int b = 0; b < nmem; ++b) {
        if (j[b] < 0) continue;
        for (int c = 0; c < j[b]; ++c)
            h[(size_t)b * ldh + c] = ws.hhost[(size_t)b * ldp + c] + ws.hhost[(size_t)(nmem + b) * ldp + c];
        beta[b] = std::sqrt(ws.hhost[(size_t)(2 * nmem + b) * ldp]);
    }
    return NSSTAB_OK;
}

// w[b] *= s[b] for members with a non-null w[b]
int scale_batch(int nmem, double* const* w, long n, const double* s, GsBatch& ws, cudaStream_t stream,
                const long* nm) {
    NS_TRY(ws.alloc(nmem, 1));
    const long* nd = nullptr;
    if (nm) {
        NS_CUDA(cudaMemcpyAsync(ws.ndev, nm, nmem * sizeof(long), cudaMemcpyHostToDevice, stream));
        nd = ws.ndev;
    }
    std::vector<double*> ph(w, w + nmem);
    NS_CUDA(cudaMemcpyAsync(ws.ptrs, ph.data(), nmem * sizeof(double*), cudaMemcpyHostToDevice, stream));
    std::vector<double> sh(s, s + nmem);
    NS_CUDA(cudaMemcpyAsync(ws.sdev, sh.data(), nmem * sizeof(double), cudaMemcpyHostToDevice, stream));
    k_scale_b<<<dim3(ws.grid, nmem), kGsThreads, 0, stream>>>(ws.ptrs, n, ws.sdev, nd);
    NS_LAUNCH_CHECK();
    return NSSTAB_OK;
}

int GsWork::alloc(int max_cols_) {
    if (max_cols_ <= max_cols) return NSSTAB_OK;
    release();
    max_cols = max_cols_;
    grid = kGsBlocks;
    NS_CUDA(cudaMalloc(&partial, (size_t)grid * max_cols * sizeof(double)));
    NS_CUDA(cudaMalloc(&hdev, (size_t)(2 * max_cols + 2) * sizeof(double)));
    NS_CUDA(cudaMallocHost(&hhost, (size_t)(2 * max_cols + 2) * sizeof(double)));
    return NSSTAB_OK;
}

void GsWork::release() {
    if (partial) cudaFree(partial);
    if (hdev) cudaFree(hdev);
    if (hhost) cudaFreeHost(hhost);
    partial = hdev = hhost = nullptr;
    max_cols = 0;
}

static int dot_into(const double* V, long ldv, long n, int j, const double* w, double* out, GsWork& ws,
                    cudaStream_t stream) {
    k_gs_dot<<<ws.grid, kGsThreads, 0, stream>>>(V, ldv, n, j, w, ws.partial, ws.max_cols);
    NS_LAUNCH_CHECK();
    k_gs_reduce_par<<<(j + 31) / 32, 256, 0, stream>>>(ws.partial, ws.grid, ws.max_cols, j, nullptr, out, 0);
    NS_LAUNCH_CHECK();
    return NSSTAB_OK;
}

static int update(double* w, const double* V, long ldv, long n, int j, const double* h, cudaStream_t stream) {
    k_gs_update<<<kGsBlocks * 2, kGsThreads, j * sizeof(double), stream>>>(w, V, ldv, n, j, h);
    NS_LAUNCH_CHECK();
    return NSSTAB_OK;
}

int cgs2(const double* V, long ldv, long n, int j, double* w, double* h, double* beta, GsWork& ws,
         cudaStream_t stream) {
    NS_TRY(ws.alloc(std::max(j, 1)));
    double* h1 = ws.hdev;
    double* h2 = ws.hdev + ws.max_cols;
    double* b2 = ws.hdev + 2 * ws.max_cols;
    if (j > 0) {
        NS_TRY(dot_into(V, ldv, n, j, w, h1, ws, stream));
        NS_TRY(update(w, V, ldv, n, j, h1, stream));
        NS_TRY(dot_into(V, ldv, n, j, w, h2, ws, stream));
        NS_TRY(update(w, V, ldv, n, j, h2, stream));
    }
    NS_TRY(dot_into(w, n, n, 1, w, b2, ws, stream));
    NS_CUDA(cudaMemcpyAsync(ws.hhost, ws.hdev, (size_t)(2 * ws.max_cols + 1) * sizeof(double),
                            cudaMemcpyDeviceToHost, stream));
    NS_CUDA(cudaStreamSynchronize(stream));
    for (int c = 0; c < j; ++c) h[c] = ws.hhost[c] + ws.hhost[ws.max_cols + c];
    *beta = std::sqrt(ws.hhost[2 * ws.max_cols]);
    return NSSTAB_OK;
}

int vec_norm(const double* x, long n, double* out, GsWork& ws, cudaStream_t stream) {
    NS_TRY(ws.alloc(1));
    double* b2 = ws.hdev + 2 * ws.max_cols;
    NS_TRY(dot_into(x, n, n, 1, x, b2, ws, stream));
    NS_CUDA(cudaMemcpyAsync(ws.hhost, b2, sizeof(double), cudaMemcpyDeviceToHost, stream));
    NS_CUDA(cudaStreamSynchronize(stream));
    *out = std::sqrt(ws.hhost[0]);
    return NSSTAB_OK;
}

int vec_axpby(double* dst, double a, const double* x, double b, const double* y, long n, cudaStream_t stream) {
    k_axpby<<<kGsBlocks, kGsThreads, 0, stream>>>(dst, a, x, b, y, n);
    NS_LAUNCH_CHECK();
    return NSSTAB_OK;
}

int vec_scale(double* dst, const double* src, long n, double s, cudaStream_t stream) {
    k_scale<<<kGsBlocks, kGsThreads, 0, stream>>>(dst, src, n, s);
    NS_LAUNCH_CHECK();
    return NSSTAB_OK;
}

int basis_combine(const double* V, long ldv, long n, int m, const double* C_dev, int p, double* out, long ldo,
                  cudaStream_t stream) {
    k_combine<<<kGsBlocks * 2, 128, 0, stream>>>(V, ldv, n, m, C_dev, m, p, out, ldo);
    NS_LAUNCH_CHECK();
    return NSSTAB_OK;
}

}  // namespace nsstab
