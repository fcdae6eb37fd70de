// cpd_tol_noalloc: the relative error Tol of a CP model without any device
// allocation, for callers that cannot call cudaMalloc.
//
// Who needs it: a host program whose device memory belongs to another
// allocator (a framework's caching pool that must account for every byte, or
// a service that reserves all memory at start-up) must not have a library
// allocate behind its back; and cudaMalloc / cudaFree can synchronise the
// device, which a latency-bound caller cannot afford in its loop. This entry
// point takes the caller's buffers and keeps its only scratch -- one pair of
// FP64 partial sums per chunk of 16 mode-1 fibers -- in a fixed array that the
// library image itself provides.
//
// The arithmetic is that of cpd_fit's kernel (x_hat from the KRP row of each
// mode-1 fiber in the factor type, (x - x_hat)^2 and x^2 accumulated in FP64,
// fixed-order reductions), reading X in its original column-major layout.
#include <cuda_bf16.h>
#include <cuda_runtime.h>

#include <string>

#include "cpd.h"
#include "cpd_device.cuh"
#include "cpd_internal.h"

namespace cpd {
void set_error(const std::string &msg);
}

using namespace cpd;

namespace {

constexpr int kTolFibers = 16;                      // mode-1 fibers per chunk
constexpr long long kTolMaxChunks = 65536;          // => at most 1,048,576 fibers

// Scratch: residual partials [0, nchunks) and ||X||^2 partials
// [kTolMaxChunks, kTolMaxChunks + nchunks), one slot per chunk (1 MiB). Every
// GPU that loads the library holds it until the process exits. Each call
// writes every slot it later reads, so nothing has to start at zero.
static __device__ __align__(256) double g_tol_scratch[2 * kTolMaxChunks];

struct TolArgs {
    int N, R;
    long long dims[kMaxModes];
    const void *A[kMaxModes];
};

template <class XT, class T>
__device__ __forceinline__ T load_elem(const XT *p) { return (T)to_float<XT>(*p); }
template <>
__device__ __forceinline__ double load_elem<double, double>(const double *p) { return *p; }

template <class T, class XT>
__global__ void __launch_bounds__(kThreads) k_tol_chunks(const TolArgs a, const XT *__restrict__ X,
                                                         long long J, long long nchunks, double *scratch)
{
    __shared__ T sz[kTolFibers * 256];
    __shared__ double red[2][kThreads / 32];
    const int R = a.R;
    const long long I0 = a.dims[0];
    const T *A0 = reinterpret_cast<const T *>(a.A[0]);
    for (long long c = blockIdx.x; c < nchunks; c += gridDim.x) {
        const long long j0 = c * kTolFibers;
        const int nfib = (J - j0) < kTolFibers ? (int)(J - j0) : kTolFibers;
        __syncthreads();
        for (int e = threadIdx.x; e < nfib * R; e += blockDim.x) {
            const int f = e / R, r = e % R;
            long long j = j0 + f;
            T z = (T)1;
            for (int k = 1; k < a.N; ++k) {
                const long long ik = j % a.dims[k];
                j /= a.dims[k];
                z = z * reinterpret_cast<const T *>(a.A[k])[ik * R + r];
            }
            sz[f * R + r] = z;
        }
        __syncthreads();
        double res = 0.0, xx = 0.0;
        for (long long i = threadIdx.x; i < I0; i += blockDim.x) {
            T xh[kTolFibers];
#pragma unroll
            for (int f = 0; f < kTolFibers; ++f) xh[f] = (T)0;
            for (int r = 0; r < R; ++r) {
                const T v = A0[i * R + r];
#pragma unroll
                for (int f = 0; f < kTolFibers; ++f) xh[f] += v * sz[f * R + r];
            }
#pragma unroll
            for (int f = 0; f < kTolFibers; ++f) {
                if (f < nfib) {
                    const T x = load_elem<XT, T>(X + (j0 + f) * I0 + i);
                    const double d = (double)(x - xh[f]);
                    res = __fma_rn(d, d, res);
                    xx = __fma_rn((double)x, (double)x, xx);
                }
            }
        }
        for (int off = 16; off >= 1; off >>= 1) {
            res += __shfl_down_sync(0xffffffffu, res, off);
            xx += __shfl_down_sync(0xffffffffu, xx, off);
        }
        if ((threadIdx.x & 31) == 0) {
            red[0][threadIdx.x >> 5] = res;
            red[1][threadIdx.x >> 5] = xx;
        }
        __syncthreads();
        if (threadIdx.x == 0) {
            double s0 = 0.0, s1 = 0.0;
            for (int w = 0; w < (int)(blockDim.x >> 5); ++w) {
                s0 += red[0][w];
                s1 += red[1][w];
            }
            scratch[c] = s0;
            scratch[kTolMaxChunks + c] = s1;
        }
    }
}

// Fixed-order fold of the chunk partials: thread q sums chunks q, q + 256,
// ... in ascending order, then a pairwise tree over the 256 threads. A tensor
// with ||X|| = 0 has no relative error: the result is then NaN.
__global__ void __launch_bounds__(kThreads) k_tol_fold(const double *scratch, long long nchunks, double *out)
{
    __shared__ double red[2][kThreads];
    double r = 0.0, x = 0.0;
    for (long long c = threadIdx.x; c < nchunks; c += kThreads) {
        r += scratch[c];
        x += scratch[kTolMaxChunks + c];
    }
    red[0][threadIdx.x] = r;
    red[1][threadIdx.x] = x;
    __syncthreads();
    for (int w = kThreads / 2; w > 0; w >>= 1) {
        if (threadIdx.x < w) {
            red[0][threadIdx.x] += red[0][threadIdx.x + w];
            red[1][threadIdx.x] += red[1][threadIdx.x + w];
        }
        __syncthreads();
    }
    if (threadIdx.x == 0) *out = red[1][0] > 0.0 ? red[0][0] / red[1][0] : __longlong_as_double(0x7ff8000000000000LL);
}

// Device address of the scratch array on the current device. Looked up on
// every call (cudaGetSymbolAddress with the calling device current), so the
// address stays right if the device's context is reset and the library's
// device code is loaded again; the first lookup on a device may load that
// code, which is why the first call should precede any stream capture.
static cpd_status scratch_address(double **out)
{
    void *p = nullptr;
    const cudaError_t e = cudaGetSymbolAddress(&p, g_tol_scratch);
    if (e != cudaSuccess || !p) {
        set_error(std::string("cudaGetSymbolAddress(scratch): ") + cudaGetErrorString(e));
        return CPD_ECUDA;
    }
    *out = static_cast<double *>(p);
    return CPD_OK;
}

}  // namespace

extern "C" cpd_status cpd_tol_noalloc(int32_t N, const int64_t *dims, int32_t R, int32_t x_dtype,
                                      const void *X, const void *const *A, double *tol_out, void *stream)
{
    if (N < 3 || N > CPD_MAX_MODES || !dims || !X || !A || !tol_out || R < 1 || R > 256 || x_dtype < 0 ||
        x_dtype > 2) {
        set_error("cpd_tol_noalloc: invalid argument (N in [3,8], R in [1,256], non-NULL buffers)");
        return CPD_EINVAL;
    }
    TolArgs a{};
    a.N = N;
    a.R = R;
    long long J = 1;
    for (int k = 0; k < N; ++k) {
        if (dims[k] < 1 || !A[k]) {
            set_error("cpd_tol_noalloc: every dim must be >= 1 and every factor non-NULL");
            return CPD_EINVAL;
        }
        a.dims[k] = dims[k];
        a.A[k] = A[k];
        // the product of the sizes of modes 2..N is bounded before it is formed
        if (k > 0) {
            if (dims[k] > kTolMaxChunks * kTolFibers / J) {
                J = kTolMaxChunks * kTolFibers + 1;   // over the limit; reported below
                break;
            }
            J *= dims[k];
        }
    }
    for (int k = 0; k < N; ++k) {
        if (dims[k] < 1 || !A[k]) {
            set_error("cpd_tol_noalloc: every dim must be >= 1 and every factor non-NULL");
            return CPD_EINVAL;
        }
    }
    const long long nchunks = (J + kTolFibers - 1) / kTolFibers;
    if (nchunks > kTolMaxChunks) {
        set_error("cpd_tol_noalloc: the tensor has more mode-1 fibers than the fixed scratch serves, at most " +
                  std::to_string(kTolMaxChunks * kTolFibers) + " (use cpd_fit)");
        return CPD_EINVAL;
    }
    double *scratch = nullptr;
    cpd_status st = scratch_address(&scratch);
    if (st != CPD_OK) return st;
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    int dev = 0, sms = 0;
    cudaError_t ea = cudaGetDevice(&dev);
    if (ea == cudaSuccess) ea = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    if (ea != cudaSuccess || sms < 1) {
        set_error(std::string("cpd_tol_noalloc: device attributes: ") + cudaGetErrorString(ea));
        return CPD_ECUDA;
    }
    const long long cap = 8LL * sms;   // eight CTAs per SM, each walking chunks
    const int grid = (int)(nchunks < cap ? nchunks : cap);
    if (x_dtype == CPD_F64)
        k_tol_chunks<double, double><<<grid, kThreads, 0, s>>>(a, (const double *)X, J, nchunks, scratch);
    else if (x_dtype == CPD_F32)
        k_tol_chunks<float, float><<<grid, kThreads, 0, s>>>(a, (const float *)X, J, nchunks, scratch);
    else
        k_tol_chunks<float, __nv_bfloat16><<<grid, kThreads, 0, s>>>(a, (const __nv_bfloat16 *)X, J, nchunks,
                                                                     scratch);
    cudaError_t e = cudaGetLastError();
    if (e == cudaSuccess) {
        k_tol_fold<<<1, kThreads, 0, s>>>(scratch, nchunks, tol_out);
        e = cudaGetLastError();
    }
    if (e != cudaSuccess) {
        set_error(std::string("cpd_tol_noalloc launch: ") + cudaGetErrorString(e));
        return CPD_ECUDA;
    }
    return CPD_OK;
}
