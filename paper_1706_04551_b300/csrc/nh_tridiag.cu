// nh_tridiag.cu -- standalone batched tridiagonal solve of the 1D pressure systems
// (App. B, Eqs. 42-43, solved by the Thomas algorithm in Sec. 4.3), exposed through the
// C-ABI for callers that assemble their own rows.
#include "../../include/nh.h"
#include "nh_internal.h"

#include <cuda_runtime.h>

namespace {

template <typename T>
int tridiag_alloc(int n, int rows, const void* a, const void* b, const void* c, const void* d,
                  void* x, cudaStream_t s)
{
    T* cp = nullptr;
    T* dp = nullptr;
    const bool need = n > nh::pcr_max_n((int)sizeof(T));
    if (need) {
        const size_t bytes = (size_t)n * rows * sizeof(T);
        if (cudaMallocAsync((void**)&cp, bytes, s) != cudaSuccess ||
            cudaMallocAsync((void**)&dp, bytes, s) != cudaSuccess) {
            cudaGetLastError();
            if (cp) cudaFreeAsync(cp, s);
            return NH_ENOMEM;
        }
    }
    int rc = nh::launch_tridiag_raw<T>(n, rows, (const T*)a, (const T*)b, (const T*)c,
                                       (const T*)d, (T*)x, cp, dp, s);
    if (need) {
        cudaFreeAsync(cp, s);
        cudaFreeAsync(dp, s);
    }
    if (rc != 0 || cudaPeekAtLastError() != cudaSuccess) {
        cudaGetLastError();
        return NH_ECUDA;
    }
    return NH_OK;
}

}  // namespace

extern "C" int nh_tridiag_batched(int n, int rows, int precision, const void* a, const void* b,
                                  const void* c, const void* d, void* x, void* stream)
{
    if (n < 2 || rows < 1 || !a || !b || !c || !d || !x) return NH_EINVAL;
    if ((double)n * (double)rows > 2.0e9) return NH_EINVAL;
    cudaStream_t s = (cudaStream_t)stream;
    if (precision == NH_FP64) return tridiag_alloc<double>(n, rows, a, b, c, d, x, s);
    if (precision == NH_FP32) return tridiag_alloc<float>(n, rows, a, b, c, d, x, s);
    return NH_EINVAL;
}

// ---------------------------------------------------------------------------------------
// Allocation-free variant.  Some callers cannot allocate device memory while they run:
// code inside another framework's memory pool or arena that forbids foreign allocations,
// work issued from callbacks or real-time loops where cudaMalloc's implicit
// synchronisation and latency are not acceptable, or processes that must keep a fixed
// device footprint.  For them the Thomas path below keeps its scratch in this file-scope
// device array instead.  It lives on every GPU that loads the library until the process
// exits.  Its address is looked up once per device with cudaGetSymbolAddress; the host
// never passes the symbol itself to a kernel.
// ---------------------------------------------------------------------------------------

#include <mutex>

namespace {

static __device__ __align__(256) unsigned char g_noalloc_scratch[NH_NOALLOC_SCRATCH_BYTES];

constexpr int kMaxDevices = 64;
std::mutex g_noalloc_mu;
void* g_noalloc_ptr[kMaxDevices] = {};

// Device address of g_noalloc_scratch on the current device (set-up on first use).
int noalloc_scratch(void** out)
{
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= kMaxDevices) {
        cudaGetLastError();
        return NH_ECUDA;
    }
    std::lock_guard<std::mutex> lock(g_noalloc_mu);
    if (!g_noalloc_ptr[dev]) {
        void* p = nullptr;
        if (cudaGetSymbolAddress(&p, g_noalloc_scratch) != cudaSuccess || !p) {
            cudaGetLastError();
            return NH_ECUDA;
        }
        g_noalloc_ptr[dev] = p;
    }
    *out = g_noalloc_ptr[dev];
    return NH_OK;
}

template <typename T>
int tridiag_noalloc(int n, int rows, const void* a, const void* b, const void* c,
                    const void* d, void* x, cudaStream_t s)
{
    T* cp = nullptr;
    T* dp = nullptr;
    if (n > nh::pcr_max_n((int)sizeof(T))) {
        const size_t half = (size_t)NH_NOALLOC_SCRATCH_BYTES / 2;
        const size_t bytes = (size_t)n * rows * sizeof(T);
        if (bytes > half) return NH_EINVAL;       // beyond the fixed scratch size
        void* base = nullptr;
        int rc = noalloc_scratch(&base);
        if (rc != NH_OK) return rc;
        cp = static_cast<T*>(base);
        dp = reinterpret_cast<T*>(static_cast<unsigned char*>(base) + half);
    }
    // Thomas writes every scratch entry before reading it, so nothing left over from an
    // earlier call is ever used and no clearing is needed.
    int rc = nh::launch_tridiag_raw<T>(n, rows, (const T*)a, (const T*)b, (const T*)c,
                                       (const T*)d, (T*)x, cp, dp, s);
    if (rc != 0 || cudaPeekAtLastError() != cudaSuccess) {
        cudaGetLastError();
        return NH_ECUDA;
    }
    return NH_OK;
}

}  // namespace

extern "C" int nh_tridiag_batched_noalloc(int n, int rows, int precision, const void* a,
                                          const void* b, const void* c, const void* d, void* x,
                                          void* stream)
{
    if (n < 2 || rows < 1 || !a || !b || !c || !d || !x) return NH_EINVAL;
    cudaStream_t s = (cudaStream_t)stream;
    if (precision == NH_FP64) return tridiag_noalloc<double>(n, rows, a, b, c, d, x, s);
    if (precision == NH_FP32) return tridiag_noalloc<float>(n, rows, a, b, c, d, x, s);
    return NH_EINVAL;
}
