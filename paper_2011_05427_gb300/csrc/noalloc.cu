// noalloc.cu -- the high-order sweep for callers that cannot allocate device memory.
//
// The paper has no counterpart to this entry point; it is a deployment convenience.
// trt_k_sweep needs a handle, and a handle needs a caller-allocated workspace.  Some
// callers cannot provide one: a plug-in hosted by an application that owns every device
// allocation and exposes no allocator to it, or a solver loop that runs after start-up
// under a fixed memory budget where a cudaMalloc (and the device-wide synchronisation it
// implies) is not allowed.  trt_sweep_noalloc takes all inputs and outputs as plain device
// pointers and keeps the sweep's scratch -- the per-direction-tile angular partial sums
// and the exit intensities -- in one file-scope static device array instead.
#include <mutex>
#include <string>
#include "common.cuh"

namespace {

// Shared by every call on a device; every GPU that loads the library holds it until exit.
static __device__ __align__(256) double g_sweep_scratch[TRT_STATIC_SCRATCH_BYTES / sizeof(double)];

std::mutex g_mu;
double *g_scratch_addr[64] = {nullptr};   // device address of g_sweep_scratch, per device
std::string g_noalloc_error;

int noalloc_fail(int code, const std::string &msg)
{
    std::lock_guard<std::mutex> lk(g_mu);
    g_noalloc_error = msg;
    return code;
}

}  // namespace

using namespace trt;

extern "C" {

size_t trt_sweep_noalloc_scratch_bytes(int nx, int N, int G)
{
    if (nx < 1 || N < 1 || G < 1) return 0;
    Problem p{};
    p.nx = nx; p.N = N; p.M = 2 * N; p.G = G; p.ldG = (G + 31) / 32 * 32;
    return sizeof(double) * (sweep_partial_doubles(p) + (size_t)p.M * p.ldG);
}

int trt_sweep_noalloc(int nx, int N, int G, int precision, double dt, const double *h,
                      const double *mu, const double *w, const double *Iin0,
                      const double *IinX, const double *sigE, const double *emis,
                      const void *I_old, void *I_new, double *f, double *fb0, double *fbX,
                      double *C0, double *CX, void *stream)
{
    if (nx < 1 || nx > 2048 || N < 1 || N > 256 || G < 1 || !(dt > 0) ||
        precision < 0 || precision > TRT_MIXED)
        return noalloc_fail(TRT_EINVAL, "trt_sweep_noalloc: bad sizes or precision");
    if (!h || !mu || !w || !Iin0 || !IinX || !sigE || !emis || !I_old || !I_new || !f || !fb0 ||
        !fbX || !C0 || !CX)
        return noalloc_fail(TRT_EINVAL, "trt_sweep_noalloc: null pointer");
    const size_t need = trt_sweep_noalloc_scratch_bytes(nx, N, G);
    if (need > TRT_STATIC_SCRATCH_BYTES)
        return noalloc_fail(TRT_ENOSPACE,
                            "trt_sweep_noalloc: problem needs " + std::to_string(need) +
                                " bytes of scratch, the static array holds " +
                                std::to_string((size_t)TRT_STATIC_SCRATCH_BYTES));
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return noalloc_fail(TRT_ECUDA, cudaGetErrorString(e));
    if (dev < 0 || dev >= 64) return noalloc_fail(TRT_ECUDA, "device index out of range");
    double *scratch;
    {
        // first call on this device: look up the array's device address (host code sees
        // only a host-side stand-in for the symbol)
        std::lock_guard<std::mutex> lk(g_mu);
        if (!g_scratch_addr[dev]) {
            double *ptr = nullptr;
            e = cudaGetSymbolAddress(reinterpret_cast<void **>(&ptr), g_sweep_scratch);
            if (e != cudaSuccess) {
                g_noalloc_error = cudaGetErrorString(e);
                return TRT_ECUDA;
            }
            g_scratch_addr[dev] = ptr;
        }
        scratch = g_scratch_addr[dev];
    }
    Problem p{};
    p.nx = nx; p.N = N; p.M = 2 * N; p.G = G; p.ldG = (G + 31) / 32 * 32;
    p.precision = precision;
    p.stream = reinterpret_cast<cudaStream_t>(stream);
    p.h = const_cast<double *>(h);
    p.mu = const_cast<double *>(mu);
    p.w = const_cast<double *>(w);
    p.Iin0 = const_cast<double *>(Iin0);
    p.IinX = const_cast<double *>(IinX);
    double *part = scratch;
    double *psi_exit = scratch + sweep_partial_doubles(p);
    e = launch_sweep(p, dt, sigE, emis, false, I_old, I_new, part, psi_exit, f, fb0, fbX, C0, CX);
    if (e != cudaSuccess) return noalloc_fail(TRT_ECUDA, cudaGetErrorString(e));
    return TRT_OK;
}

const char *trt_sweep_noalloc_error(void)
{
    std::lock_guard<std::mutex> lk(g_mu);
    return g_noalloc_error.c_str();
}

}  // extern "C"
