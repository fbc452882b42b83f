// noalloc.cu -- cross sections from caller-held DFT accumulators without any
// allocation (nlf_flux_spectra_static).
//
// The flux reduction needs one block of FP64 partial sums per frequency.
// nlf_get_spectra keeps that scratch inside the context's state; this entry
// point serves callers that hold the accumulators in their own device memory
// and cannot call cudaMalloc (a fixed memory budget owned by another
// allocator, or a loop that must not take cudaMalloc / cudaFree and their
// implicit synchronisation): the partial sums live in a fixed file-scope
// device array instead.
#include <cuda_runtime.h>

#include <mutex>

#include "../../include/nlfdtd.h"
#include "nlf_internal.h"

namespace nlf {
void launch_flux(const double2* accE, const double2* accH, const double* coef, long long n_abs, long long nrec,
                 int nf, double2* partial, int G, double dA, double* out, cudaStream_t st);
}

// Partial sums of the flux reduction: blocks x frequencies pairs of doubles.
// Every device that loads the library holds this array (2.4 MB) until exit.
static __device__ __align__(256) double2 g_flux_partial_static[NLF_FLUX_STATIC_PAIRS];

namespace {

constexpr int kMaxDevices = 64;
std::mutex g_sym_mu;
double2* g_sym_ptr[kMaxDevices] = {};

// Device address of the static array on the current device, looked up once
// per device (host code only sees a stand-in for the symbol).  The cached
// address belongs to the device's current context: after cudaDeviceReset (or
// a release and re-creation of the primary context) the module is loaded
// again and the cached address is stale, so callers that reset a device must
// not call nlf_flux_spectra_static on it again in the same process.
int static_scratch(double2** out)
{
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= kMaxDevices) return NLF_E_CUDA;
    std::lock_guard<std::mutex> lk(g_sym_mu);
    if (!g_sym_ptr[dev]) {
        void* p = nullptr;
        if (cudaGetSymbolAddress(&p, g_flux_partial_static) != cudaSuccess) return NLF_E_CUDA;
        g_sym_ptr[dev] = static_cast<double2*>(p);
    }
    *out = g_sym_ptr[dev];
    return NLF_OK;
}

}  // namespace

extern "C" int nlf_flux_spectra_static(const double* acc_e, const double* acc_h, const double* coef, long long n_abs,
                                       long long n_records, int nf, double dA, double* out, void* cuda_stream)
{
    if (!acc_e || !acc_h || !coef || !out || nf < 1 || n_records < 1 || n_abs < 0 || n_abs > n_records ||
        !(dA > 0.0))
        return NLF_E_ARG;
    if ((long long)nf > NLF_FLUX_STATIC_PAIRS) return NLF_E_ARG;
    // the same block count as the context path, capped by the static array
    long long G = n_records / 64;
    if (G < 1) G = 1;
    if (G > 608) G = 608;
    if (G * nf > NLF_FLUX_STATIC_PAIRS) G = NLF_FLUX_STATIC_PAIRS / nf;
    // an error left pending by earlier, unrelated work is reported as it
    // stands (not cleared), and nothing is launched
    if (cudaPeekAtLastError() != cudaSuccess) return NLF_E_CUDA;
    double2* partial = nullptr;
    int rc = static_scratch(&partial);
    if (rc) return rc;
    // every partial sum is written before it is read: nothing to clear
    nlf::launch_flux(reinterpret_cast<const double2*>(acc_e), reinterpret_cast<const double2*>(acc_h), coef, n_abs,
                     n_records, nf, partial, (int)G, dA, out, (cudaStream_t)cuda_stream);
    // nothing was pending before the launches: this is their own status
    return cudaGetLastError() == cudaSuccess ? NLF_OK : NLF_E_CUDA;
}
