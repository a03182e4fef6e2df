// CGS2 orthogonalisation for callers that must not allocate device memory.
//
// Some hosts of this library cannot call cudaMalloc at the point where they
// orthogonalise a vector: code inside a framework whose memory pool owns
// all device memory and forbids side allocations, or real-time loops that
// must not take the allocator's locks or risk an allocation failure in
// the middle of a run.  This entry point does the same work as
// cgs2_orthogonalize but keeps its scratch (the per-block partial dot
// products and the two coefficient vectors) in one file-scope device array
// of fixed size, so it never allocates: no cudaMalloc, cudaFree,
// cudaMallocHost or allocating library routine is called.
//
// The array exists once per GPU that loads the library and lives until the
// process exits.  Every call on a device uses the same array, so calls whose
// GPU work overlaps (on different streams, or from different host threads)
// race on it; serialise them.  The first call on a device looks up the
// array's device address once; a later reset of that device's primary
// context (cudaDeviceReset) is not supported.
#include <mutex>

#include "stepper.cuh"

namespace nsstab {

// kernels shared with krylov.cu (defined there)
__global__ void k_gs_dot(const double* __restrict__ V, long ldv, long n, int j, const double* __restrict__ w,
                         double* __restrict__ partial, int ldp);
__global__ void k_gs_reduce(const double* __restrict__ partial, int nb, int ldp, int j, double* __restrict__ out);
__global__ void k_gs_update(double* __restrict__ w, const double* __restrict__ V, long ldv, long n, int j,
                            const double* __restrict__ h);

namespace {

constexpr int kMaxCols = NSSTAB_NOALLOC_MAX_COLS;   // largest j accepted
// The grid of the dot-product kernel is fixed by the static scratch size
// (one row of partial sums per block), not by the GPU's SM count.
constexpr int kBlocks = 152;
constexpr int kThreads = 256;
// [kBlocks][kMaxCols] partials | h1 [kMaxCols] | h2 [kMaxCols] | beta^2 | h1+h2 [kMaxCols]
constexpr int kScratch = kBlocks * kMaxCols + 3 * kMaxCols + 8;

static __device__ __align__(256) double g_scratch[kScratch];

// out[c] = a[c] + b[c] for c < j
__global__ void k_sum_pair(const double* __restrict__ a, const double* __restrict__ b, double* __restrict__ out,
                           int j) {
    for (int c = threadIdx.x; c < j; c += blockDim.x) out[c] = a[c] + b[c];
}

constexpr int kMaxDevices = 64;
std::mutex g_mutex;
double* g_addr[kMaxDevices] = {nullptr};

// Device address of g_scratch on the current device, looked up once per
// device with that device current (in host code the name g_scratch is only
// a host-side stand-in, not a device address).  The cached address stays
// valid for the life of the device's primary context.
int scratch_address(double** out) {
    int dev = -1;
    NS_CUDA(cudaGetDevice(&dev));
    if (dev < 0 || dev >= kMaxDevices) {
        set_error("cgs2_orthogonalize_noalloc: device index out of range");
        return NSSTAB_ERR_INVALID_ARG;
    }
    std::lock_guard<std::mutex> lock(g_mutex);
    if (!g_addr[dev]) {
        void* p = nullptr;
        const cudaError_t e = cudaGetSymbolAddress(&p, g_scratch);
        if (e != cudaSuccess) {
            set_error(std::string("cudaGetSymbolAddress(g_scratch): ") + cudaGetErrorString(e));
            return NSSTAB_ERR_CUDA;
        }
        g_addr[dev] = static_cast<double*>(p);
    }
    *out = g_addr[dev];
    return NSSTAB_OK;
}

}  // namespace

}  // namespace nsstab

using namespace nsstab;

extern "C" int cgs2_orthogonalize_noalloc(const double* V, long ldv, long n, int j, double* w, double* h,
                                          double* beta, void* stream_) {
    if (!w || !beta || (j > 0 && (!V || !h))) {
        set_error("cgs2_orthogonalize_noalloc: null argument");
        return NSSTAB_ERR_INVALID_ARG;
    }
    if (n < 1 || j < 0 || (j > 0 && ldv < n)) {
        set_error("cgs2_orthogonalize_noalloc: bad sizes");
        return NSSTAB_ERR_INVALID_ARG;
    }
    if (j > kMaxCols) {
        set_error("cgs2_orthogonalize_noalloc: j exceeds NSSTAB_NOALLOC_MAX_COLS (256); use cgs2_orthogonalize");
        return NSSTAB_ERR_INVALID_ARG;
    }
    double* s = nullptr;
    NS_TRY(scratch_address(&s));
    cudaStream_t stream = (cudaStream_t)stream_;
    double* partial = s;
    double* h1 = s + (size_t)kBlocks * kMaxCols;
    double* h2 = h1 + kMaxCols;
    double* b2 = h2 + kMaxCols;
    double* hsum = b2 + 8;
    // every scratch entry that is read is written earlier in the same call,
    // so nothing has to be cleared between calls
    if (j > 0) {
        k_gs_dot<<<kBlocks, kThreads, 0, stream>>>(V, ldv, n, j, w, partial, kMaxCols);
        k_gs_reduce<<<1, 256, 0, stream>>>(partial, kBlocks, kMaxCols, j, h1);
        k_gs_update<<<2 * kBlocks, kThreads, j * sizeof(double), stream>>>(w, V, ldv, n, j, h1);
        k_gs_dot<<<kBlocks, kThreads, 0, stream>>>(V, ldv, n, j, w, partial, kMaxCols);
        k_gs_reduce<<<1, 256, 0, stream>>>(partial, kBlocks, kMaxCols, j, h2);
        k_gs_update<<<2 * kBlocks, kThreads, j * sizeof(double), stream>>>(w, V, ldv, n, j, h2);
        k_sum_pair<<<1, 256, 0, stream>>>(h1, h2, hsum, j);
    }
    k_gs_dot<<<kBlocks, kThreads, 0, stream>>>(w, n, n, 1, w, partial, kMaxCols);
    k_gs_reduce<<<1, 256, 0, stream>>>(partial, kBlocks, kMaxCols, 1, b2);
    NS_LAUNCH_CHECK();
    double bb = 0.0;
    if (j > 0) NS_CUDA(cudaMemcpyAsync(h, hsum, (size_t)j * sizeof(double), cudaMemcpyDeviceToHost, stream));
    NS_CUDA(cudaMemcpyAsync(&bb, b2, sizeof(double), cudaMemcpyDeviceToHost, stream));
    NS_CUDA(cudaStreamSynchronize(stream));
    *beta = std::sqrt(bb);
    return NSSTAB_OK;
}
