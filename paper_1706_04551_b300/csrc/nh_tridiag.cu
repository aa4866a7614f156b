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
