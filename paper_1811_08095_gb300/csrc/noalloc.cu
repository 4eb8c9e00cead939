// odwf_apply_m5_noalloc: the site-local M, M^dag, M^-1, M^-dag of odwf_apply_m5 for
// callers that must not allocate device memory.
//
// Some callers cannot let a library call cudaMalloc: applications whose own memory
// manager has reserved the GPU's memory up front (a framework's pool allocator holding
// most of the HBM, where a library-side cudaMalloc fails or fragments the pool), and
// latency-critical code that cannot afford the device-wide synchronisation that
// cudaMalloc / cudaFree imply.  odwf_apply_m5 stages its input and result in internal
// layout in workspaces it allocates on first use; this variant stages them in a
// fixed file-scope device array instead and needs no handle, so it allocates nothing.
//
// The array holds the FP64 mass parameter r and two packed fields of at most
// kNoAllocMaxSites5 = 65,536 five-dimensional sites (n_sites x Ns): 24 MiB + 256 B that
// every GPU which loads the library keeps until the process exits.  Host code reaches
// it only through the address that cudaGetSymbolAddress returns for the current device
// (the array's name in host code is a host-side stand-in, not a device address); that
// look-up happens on the first call on each device, with the device current.  Under CUDA's
// lazy module loading (the default) the array is reserved when this file's module is first
// used on a device -- that same first call -- not when the library is loaded; with
// CUDA_MODULE_LOADING=EAGER it is reserved when the device's context is created.
#include <cmath>
#include <cstring>
#include <mutex>
#include <string>

#include "../../include/odwf.h"
#include "kernels.cuh"
#include "kernels.h"

namespace odwf {

int fail(int code, const std::string& msg);
bool is_device_ptr(const void* p);
int check_ptr_device(const void* p, int dev, const char* what);

namespace {

constexpr size_t kNoAllocMaxSites5 = 65536;
constexpr size_t kFieldBytes = kNoAllocMaxSites5 * 192;  // one FP64 packed field
constexpr size_t kScratchBytes = 256 + 2 * kFieldBytes;   // r (padded to 256 B) + input + result

static __device__ __align__(256) unsigned char g_noalloc_scratch[kScratchBytes];

constexpr int kMaxDevices = 64;
std::mutex g_mu;
unsigned char* g_scratch_addr[kMaxDevices] = {nullptr};

__global__ void set_r_kernel(double* dst, double r) { *dst = r; }

// Device address of the scratch array for the current device (looked up once per device).
int scratch_for_current_device(unsigned char** out) {
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return fail(ODWF_ECUDA, std::string("odwf_apply_m5_noalloc: cudaGetDevice: ") +
                                                      cudaGetErrorString(e));
    if (dev < 0 || dev >= kMaxDevices) return fail(ODWF_EINVAL, "odwf_apply_m5_noalloc: device index out of range");
    std::lock_guard<std::mutex> g(g_mu);
    if (!g_scratch_addr[dev]) {
        void* p = nullptr;
        e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
        if (e != cudaSuccess || !p)
            return fail(ODWF_ECUDA, std::string("odwf_apply_m5_noalloc: cudaGetSymbolAddress: ") +
                                        cudaGetErrorString(e));
        g_scratch_addr[dev] = (unsigned char*)p;
    }
    *out = g_scratch_addr[dev];
    return ODWF_OK;
}

}  // namespace

}  // namespace odwf

using odwf::fail;

extern "C" int odwf_apply_m5_noalloc(int Ns, double m0, double mq, const double* omega, void* out, const void* in,
                                     long n_sites, int op, void* stream) {
    using namespace odwf;
    if (!omega || !out || !in) return fail(ODWF_EINVAL, "odwf_apply_m5_noalloc: null argument");
    if (Ns < 2 || Ns > kMaxNs || (Ns & (Ns - 1)))
        return fail(ODWF_EINVAL, "odwf_apply_m5_noalloc: Ns must be 2, 4, 8, 16 or 32");
    if (op < 0 || op > 3) return fail(ODWF_EINVAL, "odwf_apply_m5_noalloc: op must be 0..3");
    if (n_sites <= 0 || n_sites > (long)(kNoAllocMaxSites5 / (size_t)Ns))
        return fail(ODWF_EINVAL, "odwf_apply_m5_noalloc: n_sites x Ns must be between 1 and 65536 "
                                 "(the size of the library's fixed scratch array)");
    if (!(m0 != 0.0) || !std::isfinite(m0) || !std::isfinite(mq))
        return fail(ODWF_EINVAL, "odwf_apply_m5_noalloc: bad m0 or mq");
    if (!is_device_ptr(in) || !is_device_ptr(out))
        return fail(ODWF_EINVAL, "odwf_apply_m5_noalloc: in and out must be device memory");
    {
        int dev = 0;
        const cudaError_t e = cudaGetDevice(&dev);
        if (e != cudaSuccess)
            return fail(ODWF_ECUDA, std::string("odwf_apply_m5_noalloc: cudaGetDevice: ") + cudaGetErrorString(e));
        int rc0 = check_ptr_device(in, dev, "odwf_apply_m5_noalloc (in)");
        if (!rc0) rc0 = check_ptr_device(out, dev, "odwf_apply_m5_noalloc (out)");
        if (rc0) return rc0;
    }
    // coefficients of M = (4 - m0) B + 1 - L, B = rho + sigma L, rho = sigma = omega (kernel parameters)
    Coef5<double> cf;
    std::memset(&cf, 0, sizeof(cf));
    const double a = 4.0 - m0;
    for (int s = 0; s < Ns; ++s) {
        if (!std::isfinite(omega[s])) return fail(ODWF_EINVAL, "odwf_apply_m5_noalloc: non-finite omega");
        cf.rho[s] = cf.sigma[s] = omega[s];
        cf.d[s] = a * omega[s] + 1.0;
        cf.e[s] = a * omega[s] - 1.0;
        if (cf.d[s] == 0.0) return fail(ODWF_EINVAL, "odwf_apply_m5_noalloc: singular diagonal");
        cf.inv_d[s] = 1.0 / cf.d[s];
    }
    unsigned char* base = nullptr;
    int rc = scratch_for_current_device(&base);
    if (rc) return rc;
    double* r_dev = (double*)base;
    FieldRef X{base + 256, nullptr, 0, 0};
    FieldRef Y{base + 256 + kFieldBytes, nullptr, 0, 0};
    cudaStream_t st = (cudaStream_t)stream;
    Geom gf;
    std::memset(&gf, 0, sizeof(gf));
    gf.Vh = (int)n_sites;  // a flat list of sites
    const int lg = lg2(Ns);
    const int bs = 256;
    const int grid = blocks_for((size_t)n_sites * Ns, bs);
    // every byte read below is written first in the same stream: nothing relies on zeroed scratch
    note_launch();
    set_r_kernel<<<1, 1, 0, st>>>(r_dev, mq / (2.0 * m0));
    note_launch();
    pack_kernel<SpF64><<<grid, bs, 0, st>>>((const double2*)in, X, gf, 0, Ns, lg, 1);
    note_launch();
    m5_kernel<SpF64, SpF64, double><<<dim3(grid, 1), bs, 0, st>>>(X, Y, (size_t)n_sites, Ns, lg, r_dev, 0, op, cf, nullptr, 0);
    note_launch();
    unpack_kernel<SpF64><<<grid, bs, 0, st>>>(Y, (double2*)out, gf, 0, Ns, lg, 1);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess)
        return fail(ODWF_ECUDA, std::string("odwf_apply_m5_noalloc: launch failed: ") + cudaGetErrorString(e));
    return ODWF_OK;
}
