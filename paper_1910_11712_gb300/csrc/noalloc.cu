// nep_jacobi_svd_noalloc: the one-sided Jacobi SVD of nep_jacobi_svd, for callers that must
// not allocate device memory. Examples: a host application that hands the library a fixed
// memory budget and accounts for every device byte itself, or a real-time loop that may not
// enter the CUDA allocator (whose calls can block or synchronise) once it is running. The
// ordinary entry point obtains its work arrays from the stream-ordered allocator on every
// call; this one uses a fixed block of device memory compiled into the library instead.
//
// The block is a file-scope static __device__ array. Every GPU that loads the library holds
// it (NEP_NOALLOC_SCRATCH_BYTES) until the process exits. Host code cannot use the array's
// name as a device address: the name refers to a host-side stand-in. The device address is
// obtained once per device with cudaGetSymbolAddress, with that device current, on the first
// call made on that device.
#include <mutex>

#include "nep_common.cuh"

namespace nep {

// Layout: [256-byte control words][Vm: cols*cols complex128][U: rows*cols complex128]
constexpr size_t NOALLOC_CTRL_BYTES = 256;
constexpr size_t NOALLOC_MAX_ELEMS = 131072;  // complex128 elements for Vm + U (2 MiB)
constexpr size_t NOALLOC_SCRATCH_BYTES = NOALLOC_CTRL_BYTES + NOALLOC_MAX_ELEMS * sizeof(zd);

static __device__ __align__(256) unsigned char g_nep_noalloc_scratch[NOALLOC_SCRATCH_BYTES];

constexpr int NOALLOC_MAX_DEVICES = 64;
static void* g_scratch_addr[NOALLOC_MAX_DEVICES] = {};
static std::mutex g_scratch_mutex;

// Device address of the static block on the current device (looked up once per device).
static int scratch_address(void** out) {
    int dev = 0;
    NEP_CUDA(cudaGetDevice(&dev));
    if (dev < 0 || dev >= NOALLOC_MAX_DEVICES) {
        set_error("nep_jacobi_svd_noalloc: device ordinal %d is beyond the supported %d", dev, NOALLOC_MAX_DEVICES);
        return NEP_ERR_UNSUPPORTED;
    }
    std::lock_guard<std::mutex> lock(g_scratch_mutex);
    if (!g_scratch_addr[dev]) {
        void* p = nullptr;
        const cudaError_t e = cudaGetSymbolAddress(&p, g_nep_noalloc_scratch);
        if (e != cudaSuccess || !p) return cuda_fail(e, "cudaGetSymbolAddress(g_nep_noalloc_scratch)", __FILE__, __LINE__);
        g_scratch_addr[dev] = p;
    }
    *out = g_scratch_addr[dev];
    return NEP_OK;
}

}  // namespace nep

using namespace nep;

extern "C" int nep_jacobi_svd_noalloc(int32_t rows, int32_t cols, double* A_dev, double* W_dev, double* sigma_dev,
                                      void* stream) {
    if (rows < cols || cols < 1 || !A_dev || !W_dev || !sigma_dev) {
        set_error("nep_jacobi_svd_noalloc: need rows >= cols >= 1 and non-NULL A, W, sigma");
        return NEP_ERR_ARG;
    }
    const size_t need = (size_t)rows * cols + (size_t)cols * cols;
    if (need > NOALLOC_MAX_ELEMS) {
        set_error("nep_jacobi_svd_noalloc: rows*cols + cols*cols = %zu exceeds the fixed scratch of %zu complex "
                  "elements (e.g. 256 x 256); use nep_jacobi_svd",
                  need, NOALLOC_MAX_ELEMS);
        return NEP_ERR_ARG;
    }
    cudaStream_t st = (cudaStream_t)stream;
    void* base = nullptr;
    NEP_TRY(scratch_address(&base));
    unsigned char* b = static_cast<unsigned char*>(base);
    JacobiWork w{};
    w.flags = reinterpret_cast<int*>(b);           // 2 ints
    w.sweeps = reinterpret_cast<int*>(b + 16);     // 1 int
    w.bar = reinterpret_cast<unsigned*>(b + 32);   // 2 unsigned
    w.err = reinterpret_cast<int*>(b + 48);        // 1 int
    w.Vm = reinterpret_cast<zd*>(b + NOALLOC_CTRL_BYTES);
    zd* U = w.Vm + (size_t)cols * cols;
    // the block keeps whatever the previous call left: the control words must start at zero
    NEP_CUDA(cudaMemsetAsync(b, 0, NOALLOC_CTRL_BYTES, st));
    NEP_TRY(jacobi_svd(rows, cols, (zd*)A_dev, U, (zd*)W_dev, sigma_dev, w, st));
    NEP_CUDA(cudaMemcpyAsync(A_dev, U, sizeof(zd) * (size_t)rows * cols, cudaMemcpyDeviceToDevice, st));
    int err = 0;
    NEP_CUDA(cudaMemcpyAsync(&err, w.err, sizeof(int), cudaMemcpyDeviceToHost, st));
    NEP_CUDA(cudaStreamSynchronize(st));
    if (err) {
        set_error("nep_jacobi_svd_noalloc: a bounded grid barrier timed out");
        return NEP_ERR_INTERNAL;
    }
    return NEP_OK;
}
