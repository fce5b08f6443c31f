// noalloc.cu -- the high-order sweep for callers that cannot allocate device memory.
//
// The paper has no counterpart to this entry point; it is a deployment convenience.
// trt_k_sweep needs a handle, and a handle needs a caller-allocated workspace.  Some
// callers cannot provide one: a plug-in hosted by an application that owns every device
// allocation and exposes no allocator to it, or a solver loop that runs after start-up
// under a fixed memory budget where a cudaMalloc (and the device-wide synchronisation it
// implies) is not allowed.  trt_sweep_noalloc takes all inputs and outputs as plain device
// pointers and keeps the sweep's scratch -- the per-direction-tile angular partial sums,
// the exit intensities and, for FP32 sweeps, the pre-scaled FP32 inputs -- in one
// file-scope static device array instead.
#include <mutex>
#include <string>
#include "common.cuh"

namespace {

// Shared by every call on a device; every GPU that loads the library holds it until exit.
static __device__ __align__(256) double g_sweep_scratch[TRT_STATIC_SCRATCH_BYTES / sizeof(double)];

std::mutex g_mu;                          // guards the per-device address table
double *g_scratch_addr[64] = {nullptr};   // device address of g_sweep_scratch, per device
thread_local std::string g_noalloc_error;   // this thread's last failure

int noalloc_fail(int code, const std::string &msg)
{
    g_noalloc_error = msg;
    return code;
}

size_t al256(size_t b) { return (b + 255) / 256 * 256; }

// carve-up of the static array (byte offsets): the sweep's partial moments and exit
// intensities (both precisions), then for FP32 sweeps the per-direction FP32 constants and
// the pre-scaled FP32 inputs (sigma_t h/2, h e/2 per (group, cell), h/(2 c dt) per cell)
struct Carve {
    size_t part, psi, dir32, sig32, emis32, total;
    explicit Carve(const trt::Problem &p)
    {
        part = 0;
        psi = part + al256(sizeof(double) * trt::sweep_partial_doubles(p));
        dir32 = psi + al256(sizeof(double) * (size_t)p.M * p.ldG);
        sig32 = dir32 + al256(sizeof(float) * 4 * (size_t)p.M);
        emis32 = sig32 + al256(sizeof(float) * (size_t)p.G * p.nx);
        total = emis32 + al256(sizeof(float) * ((size_t)p.G * p.nx + p.nx));
    }
};

trt::Problem make_problem(int nx, int N, int G, int precision)
{
    trt::Problem p{};
    p.nx = nx; p.N = N; p.M = 2 * N; p.G = G; p.ldG = (G + 31) / 32 * 32;
    p.precision = precision;
    return p;
}

// the FP32 sweeps' per-direction constants |mu|, |mu|/2, w/2, w mu^2/2, each formed in FP64
// and rounded once (the operations and order of the handle's table)
__global__ void k_dir32(int M, const double *__restrict__ mu, const double *__restrict__ w,
                        float *__restrict__ dir32)
{
    const int m = blockIdx.x * blockDim.x + threadIdx.x;
    if (m >= M) return;
    const double am = fabs(mu[m]);
    dir32[4 * m + 0] = __double2float_rn(am);
    dir32[4 * m + 1] = __double2float_rn(__dmul_rn(0.5, am));
    dir32[4 * m + 2] = __double2float_rn(__dmul_rn(0.5, w[m]));
    dir32[4 * m + 3] = __double2float_rn(__dmul_rn(__dmul_rn(__dmul_rn(0.5, w[m]), mu[m]), mu[m]));
}

}  // namespace

using namespace trt;

extern "C" {

size_t trt_sweep_noalloc_scratch_bytes(int nx, int N, int G)
{
    if (nx < 1 || N < 1 || G < 1) return 0;
    return Carve(make_problem(nx, N, G, TRT_SWEEP_FP32)).total;
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
    unsigned char *scratch;
    {
        // first call on this device: look up the array's device address (host code sees
        // only a host-side stand-in for the symbol)
        std::lock_guard<std::mutex> lk(g_mu);
        if (!g_scratch_addr[dev]) {
            double *ptr = nullptr;
            e = cudaGetSymbolAddress(reinterpret_cast<void **>(&ptr), g_sweep_scratch);
            if (e != cudaSuccess) return noalloc_fail(TRT_ECUDA, cudaGetErrorString(e));
            g_scratch_addr[dev] = ptr;
        }
        scratch = reinterpret_cast<unsigned char *>(g_scratch_addr[dev]);
    }
    Problem p = make_problem(nx, N, G, precision);
    const Carve c(p);
    p.stream = reinterpret_cast<cudaStream_t>(stream);
    p.h = const_cast<double *>(h);
    p.mu = const_cast<double *>(mu);
    p.w = const_cast<double *>(w);
    p.Iin0 = const_cast<double *>(Iin0);
    p.IinX = const_cast<double *>(IinX);
    double *part = reinterpret_cast<double *>(scratch + c.part);
    double *psi_exit = reinterpret_cast<double *>(scratch + c.psi);
    if (sweep_fp32(precision)) {
        // as trt_k_sweep on an FP32 handle: the FP32 direction constants, the pre-scaled
        // FP32 inputs, then the FP32 sweep on them (every value is written before it is read)
        p.dir32 = reinterpret_cast<float *>(scratch + c.dir32);
        float *sig32 = reinterpret_cast<float *>(scratch + c.sig32);
        float *emis32 = reinterpret_cast<float *>(scratch + c.emis32);
        k_dir32<<<(p.M + 127) / 128, 128, 0, p.stream>>>(p.M, mu, w, p.dir32);
        e = cudaGetLastError();
        if (e == cudaSuccess) e = launch_prescale32(p, dt, sigE, emis, sig32, emis32);
        if (e == cudaSuccess)
            e = launch_sweep(p, dt, sig32, emis32, true, I_old, I_new, part, psi_exit, f, fb0,
                             fbX, C0, CX);
    } else {
        e = launch_sweep(p, dt, sigE, emis, false, I_old, I_new, part, psi_exit, f, fb0, fbX, C0,
                         CX);
    }
    if (e != cudaSuccess) return noalloc_fail(TRT_ECUDA, cudaGetErrorString(e));
    return TRT_OK;
}

const char *trt_sweep_noalloc_error(void)
{
    return g_noalloc_error.c_str();
}

}  // extern "C"
