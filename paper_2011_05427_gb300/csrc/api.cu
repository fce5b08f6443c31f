// api.cu -- the C ABI of include/trt.h: problem set-up, workspace carving, the Algorithm 3
// driver (one implicit time step), state access, and kernel-level entry points.
//
// Algorithm 3 (Sec. 4) as driven here, per time step j:
//   s = 0: a low-order phase with the previous step's QD factors (no sweep);
//   s > 0: opacities at T^(s) -> HO sweep -> f_g, C_g^+- -> low-order phase;
//   low-order phase: at most l_max cycles; a cycle is the fine-grid spectrum at T^(l,s)
//   followed by one grey LOQD + MEB Newton step per grid visit: first from the fine grid
//   (k = 0), then for every gamma_k of the schedule S re-evaluate the fine opacities at
//   T~^[k], restrict fine -> gamma_k, solve the coarse-group system, restrict -> grey.
// Readings (the paper is silent or garbled): the outer loop ends when BOTH the change of T
// and of the grey E are below eps (relative, infinity norm); the inner loop leaves early
// on eps_inner; T~^[0] = T^(l,s); the step ends with T of the last grey solve, E_g / F_g of
// the last fine solve and I of the last sweep; the secant derivative of the grey opacity
// restarts at zero with every time step.
// The cycles of a phase are enqueued together: the last grey visit of each cycle tests the
// inner criterion on the device and gates the cycles after it, and the host reads the
// convergence flags once per phase (one stream sync per phase).
#include <algorithm>
#include <chrono>
#include <cmath>
#include <cstdio>
#include <cstring>
#include <memory>
#include <string>
#include <vector>
#include "handle.cuh"
#include "../../include/trt_mlp.h"

using namespace trt;

static std::string g_create_error = "";


namespace {

struct Carver {
    char *base;
    size_t off;
    template <class T>
    T *take(size_t n)
    {
        off = (off + 255) / 256 * 256;
        T *ptr = base ? reinterpret_cast<T *>(base + off) : nullptr;
        off += std::max<size_t>(n, 1) * sizeof(T);
        return ptr;
    }
};

void carve_level(Carver &c, Level &L, int n, int nx)
{
    L.n = n;
    L.fine = 0;
    size_t cn = (size_t)n * nx, fn = (size_t)n * (nx + 1);
    L.phi = c.take<double>(cn); L.sig = c.take<double>(cn); L.emis = c.take<double>(cn);
    L.Eold = c.take<double>(cn); L.Esum = c.take<double>(cn); L.E = c.take<double>(cn);
    L.sigR = c.take<double>(fn); L.etaR = c.take<double>(fn); L.etaL = c.take<double>(fn);
    L.Fold = c.take<double>(fn); L.F = c.take<double>(fn);
    L.phib0 = c.take<double>(n); L.phibX = c.take<double>(n); L.C0 = c.take<double>(n);
    L.CX = c.take<double>(n); L.Ein0 = c.take<double>(n); L.Fin0 = c.take<double>(n);
    L.EinX = c.take<double>(n); L.FinX = c.take<double>(n); L.Eb0 = c.take<double>(n);
    L.EbX = c.take<double>(n);
}

void carve(trt_handle *h, Carver &c)
{
    Problem &p = h->p;
    const size_t nx = p.nx, G = p.G, M = p.M;
    const size_t rsz = sweep_fp32(p.precision) ? sizeof(float) : sizeof(double);
    p.h = c.take<double>(nx); p.edges = c.take<double>(G + 1);
    p.mu = c.take<double>(M); p.w = c.take<double>(M);
    p.Iin0 = c.take<double>(G); p.IinX = c.take<double>(G);
    p.Ein0 = c.take<double>(G); p.Fin0 = c.take<double>(G);
    p.EinX = c.take<double>(G); p.FinX = c.take<double>(G);
    p.ihf = c.take<double>(nx + 1);
    p.hf = c.take<double>(nx + 1);
    p.hc = c.take<double>(nx); p.h2 = c.take<double>(nx);
    p.fwl = c.take<double>(nx + 1); p.fwr = c.take<double>(nx + 1);
    p.hidt = c.take<double>(nx); p.dxicdt = c.take<double>(nx + 1);
    p.cterm = c.take<double>(8 * nx);   // [7][nx] doubles, nx floats, nx ints
    p.lo_dt = 0.0;
    p.dir32 = reinterpret_cast<float *>(c.take<double>(2 * M));
    p.e2tab = c.take<double>(32);
    p.lo_slot = reinterpret_cast<int *>(c.take<double>((nx + 2) / 2));
    p.otab = c.take<double>(otab_doubles((int)G));
    p.otabp = lo_pair(p.precision) ? c.take<double>(otab_doubles((int)G) + G + 1) : nullptr;
    p.cpair = lo_pair(p.precision) ? c.take<double>(5 * nx) : nullptr;
    p.lopc = lo_pair(p.precision) ? c.take<double>(8 * (nx + 1)) : nullptr;
    p.rscratch_doubles = restrict_scratch_doubles((int)nx, (int)G, 1);
    p.rscratch = p.rscratch_doubles ? c.take<double>(p.rscratch_doubles) : nullptr;
    double **tl[] = {&h->T, &h->Told, &h->Tcyc, &h->Tphase, &h->Ttil, &h->Tnew, &h->sig_prev,
                     &h->T_prev, &h->Ecyc, &h->Ephase};
    for (double **q : tl) *q = c.take<double>(nx);
    h->Eg = c.take<double>(G * nx); h->Eg_old = c.take<double>(G * nx);
    h->Fg = c.take<double>(G * (nx + 1)); h->Fg_old = c.take<double>(G * (nx + 1));
    const size_t nI = M * nx * 2 * (size_t)p.ldG;
    h->I_cur = c.take<char>(nI * rsz); h->I_alt = c.take<char>(nI * rsz);
    h->f = c.take<double>(G * nx);
    h->fb0 = c.take<double>(G); h->fbX = c.take<double>(G);
    h->C0 = c.take<double>(G); h->CX = c.take<double>(G);
    h->sigE = c.take<double>(G * nx); h->emis = c.take<double>(G * nx);
    h->sigR = c.take<double>(G * nx);
    if (sweep_fp32(p.precision)) {
        h->sig32 = c.take<float>(G * nx);
        h->emis32 = c.take<float>(G * nx + nx);   // then h/(2 c dt) per cell (kap32)
    } else {   // the paired FP64 sweep's t, s and pre-scaled inputs
        p.ts64 = c.take<double>((size_t)p.N * nx * 2 * p.ldG);
        p.tab64 = c.take<double>(2 * nx * (size_t)p.ldG + nx);
    }
    h->part = c.take<double>(std::max(sweep_partial_doubles(p), 4 * nx + 8));
    h->psi_exit = c.take<double>(M * (size_t)p.ldG);
    h->E1 = c.take<double>(G * nx); h->F1 = c.take<double>(G * (nx + 1));
    h->Eb0_1 = c.take<double>(G); h->EbX_1 = c.take<double>(G);
    h->gpre = c.take<double>(3 * nx);
    int n2 = (p.nlev >= 3) ? p.levels[1] : 1;
    carve_level(c, h->crs, n2, p.nx);
    carve_level(c, h->grey, 1, p.nx);
    h->flags = c.take<double>(10);
    h->ctl = reinterpret_cast<int *>(h->flags + 8);
}

bool validate(const trt_grid *grid, const trt_angles *angles, const trt_groups *groups,
              const trt_options *opt, Problem &p, std::vector<double> &xe,
              std::vector<double> &edges, std::string &err)
{
    if (!grid || !angles || !groups || !opt) { err = "null argument"; return false; }
    p.nx = grid->n_cells;
    if (p.nx < 1 || p.nx > 2048) { err = "n_cells must be in [1, 2048]"; return false; }
    p.N = angles->N;
    if (p.N < 1 || p.N > 256) { err = "angles.N must be in [1, 256]"; return false; }
    p.M = 2 * p.N;
    p.G = groups->n_groups;
    if (p.G < 1 || p.G > (1 << 16)) { err = "n_groups must be in [1, 65536]"; return false; }
    p.ldG = (p.G + 31) / 32 * 32;
    p.precision = opt->precision;
    if (!precision_ok(p.precision)) { err = "bad precision"; return false; }
    xe.resize(p.nx + 1);
    if (grid->x_edges) {
        for (int i = 0; i <= p.nx; ++i) xe[i] = grid->x_edges[i];
    } else {
        if (!(grid->length_cm > 0)) { err = "length_cm must be > 0"; return false; }
        for (int i = 0; i <= p.nx; ++i) xe[i] = grid->length_cm * i / p.nx;
    }
    for (int i = 0; i < p.nx; ++i)
        if (!(xe[i + 1] > xe[i])) { err = "x_edges must increase"; return false; }
    edges.resize(p.G + 1);
    if (groups->edges_keV) {
        for (int g = 0; g <= p.G; ++g) edges[g] = groups->edges_keV[g];
    } else {
        if (p.G < 3 || !(groups->nu_a > 0) || !(groups->nu_b > groups->nu_a)) {
            err = "default group edges need n_groups >= 3 and 0 < nu_a < nu_b";
            return false;
        }
        edges[0] = 0.0;
        for (int k = 0; k <= p.G - 2; ++k)
            edges[k + 1] = groups->nu_a * std::pow(groups->nu_b / groups->nu_a, (double)k / (p.G - 2));
        edges[p.G] = INFINITY;
    }
    if (!(edges[0] >= 0)) { err = "group edges must be >= 0"; return false; }
    for (int g = 0; g < p.G; ++g)
        if (!(edges[g + 1] > edges[g])) { err = "group edges must increase"; return false; }
    if (groups->level_groups && groups->n_levels >= 2) {
        p.nlev = groups->n_levels;
        if (p.nlev > 16) { err = "at most 16 grids"; return false; }
        for (int l = 0; l < p.nlev; ++l) p.levels[l] = groups->level_groups[l];
    } else if (!groups->level_groups && groups->n_levels == 0) {
        p.nlev = 2;
        p.levels[0] = p.G;
        p.levels[1] = 1;
    } else {
        err = "level_groups must list n_levels >= 2 grids";
        return false;
    }
    if (p.levels[0] != p.G || p.levels[p.nlev - 1] != 1) {
        err = "grids must run from n_groups down to 1";
        return false;
    }
    for (int l = 1; l < p.nlev; ++l)
        if (p.levels[l] < 1 || p.levels[l] > p.levels[l - 1] || p.levels[l - 1] % p.levels[l]) {
            err = "each grid must divide the previous one (uniform coarsening)";
            return false;
        }
    if (!(opt->T0_keV > 0)) { err = "T0 must be > 0"; return false; }
    p.T0 = opt->T0_keV;
    p.Tl = grid->T_left_keV;
    p.Tr = grid->T_right_keV;
    p.nu_first = edges[0];
    p.nu_last = edges[p.G];
    p.stream = reinterpret_cast<cudaStream_t>(opt->stream);
    return true;
}

__global__ void k_f_from_mlp(long n, const float *__restrict__ y, double *__restrict__ f)
{
    const long i = (long)blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n) f[i] = (double)y[i];
}

cudaError_t launch_f_from_mlp(const Problem &p, const float *y, double *f)
{
    const long n = (long)p.G * p.nx;
    k_f_from_mlp<<<(unsigned)((n + 255) / 256), 256, 0, p.stream>>>(n, y, f);
    return cudaGetLastError();
}

// Start of a low-order phase of Algorithm 3: the references of its convergence tests
// (Tphase = Tcyc = T; Ephase, Ecyc = the grey E of the phase before, or Ephase as it is in
// the step's first phase) and the inner-loop gate opened.
__global__ void k_phase_start(int nx, int from_grey, const double *__restrict__ T,
                              const double *__restrict__ Egrey, double *Tphase, double *Tcyc,
                              double *Ephase, double *Ecyc, int *ctl)
{
    griddep_wait();
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i < nx) {
        const double t = T[i];
        const double e = from_grey ? Egrey[i] : Ephase[i];
        Tphase[i] = t;
        Tcyc[i] = t;
        Ephase[i] = e;
        Ecyc[i] = e;
    }
    if (i == 0) ctl[0] = 0;
}

cudaError_t launch_phase_start(const trt_handle *h, bool from_grey)
{
    const int nx = h->p.nx;
    return launch_pdl(k_phase_start, dim3((nx + 255) / 256), dim3(256), 0, h->p.stream, nx,
                      from_grey ? 1 : 0, (const double *)h->T, (const double *)h->grey.E,
                      h->Tphase, h->Tcyc, h->Ephase, h->Ecyc, h->ctl);
}

template <typename R>
__global__ void k_fill_intensity(R *I, const double *B, long rows, int ldG, int G)
{
    long idx = (long)blockIdx.x * blockDim.x + threadIdx.x;
    long n = rows * ldG;
    for (; idx < n; idx += (long)gridDim.x * blockDim.x) {
        int g = (int)(idx % ldG);
        I[idx] = (g < G) ? (R)B[g] : (R)0;
    }
}

Level from_abi(const trt_level *l)
{
    Level L;
    L.n = l->n;
    L.fine = l->fine ? 1 : 0;
    L.phi = l->phi; L.sig = l->sig; L.emis = l->emis; L.Eold = l->Eold; L.Esum = l->Esum;
    L.sigR = l->sigR; L.etaR = l->etaR; L.etaL = l->etaL; L.Fold = l->Fold;
    L.phib0 = l->phib0; L.phibX = l->phibX; L.C0 = l->C0; L.CX = l->CX;
    L.Ein0 = l->Ein0; L.Fin0 = l->Fin0; L.EinX = l->EinX; L.FinX = l->FinX;
    L.E = l->E; L.F = l->F; L.Eb0 = l->Eb0; L.EbX = l->EbX;
    return L;
}

int fail(trt_handle *h, int code, const std::string &msg)
{
    if (h) h->err = msg;
    else g_create_error = msg;
    return code;
}

#define CK(call)                                                                           \
    do {                                                                                   \
        cudaError_t e__ = (call);                                                          \
        if (e__ != cudaSuccess)                                                            \
            return fail(h, TRT_ECUDA, std::string(#call) + ": " + cudaGetErrorString(e__)); \
    } while (0)

cudaError_t d2d(trt_handle *h, double *dst, const double *src, size_t n)
{
    return cudaMemcpyAsync(dst, src, n * sizeof(double), cudaMemcpyDeviceToDevice, h->p.stream);
}

}  // namespace

extern "C" {

size_t trt_workspace_bytes(const trt_grid *grid, const trt_angles *angles,
                           const trt_groups *groups, const trt_options *opt)
{
    trt_handle tmp{};
    std::vector<double> xe, ed;
    std::string err;
    if (!validate(grid, angles, groups, opt, tmp.p, xe, ed, err)) return 0;
    Carver c{nullptr, 0};
    carve(&tmp, c);
    return (c.off + 255) / 256 * 256;
}

int trt_create(const trt_grid *grid, const trt_angles *angles, const trt_groups *groups,
               const trt_opacity *opacity, double cv, const trt_options *opt, trt_handle **out)
{
    if (!out) return fail(nullptr, TRT_EINVAL, "out is null");
    *out = nullptr;
    (void)cudaGetLastError();   // an error left by another library is not ours to report
    trt_handle *h = nullptr;   // errors during creation go to the global message (CK)
    std::unique_ptr<trt_handle> hp(new trt_handle());
    std::vector<double> xe, edges;
    std::string err;
    if (!validate(grid, angles, groups, opt, hp->p, xe, edges, err))
        return fail(nullptr, TRT_EINVAL, err);
    if (!opacity || !(opacity->scale > 0)) return fail(nullptr, TRT_EINVAL, "opacity scale must be > 0");
    if (!(cv > 0)) return fail(nullptr, TRT_EINVAL, "cv must be > 0");
    Problem &p = hp->p;
    p.s = opacity->scale;
    p.tr_mode = opacity->tr_mode ? 1 : 0;
    p.cv = cv;
    Carver dry{nullptr, 0};
    carve(hp.get(), dry);
    const size_t need = (dry.off + 255) / 256 * 256;
    if (!opt->workspace || (reinterpret_cast<uintptr_t>(opt->workspace) & 255))
        return fail(nullptr, TRT_EINVAL, "workspace must be a 256-byte aligned device pointer");
    if (opt->workspace_bytes < need)
        return fail(nullptr, TRT_ENOSPACE, "workspace too small: need " + std::to_string(need) +
                                               " bytes");
    {
        cudaError_t e = ensure_tables();
        if (e != cudaSuccess) return fail(nullptr, TRT_ECUDA, cudaGetErrorString(e));
    }
    Carver c{reinterpret_cast<char *>(opt->workspace), 0};
    trt_handle *H = hp.get();
    carve(H, c);
    {
        cudaError_t e = cudaMallocHost(&H->hflags, 10 * sizeof(double));
        if (e != cudaSuccess) return fail(nullptr, TRT_ECUDA, cudaGetErrorString(e));
        e = cudaEventCreateWithFlags(&H->ev_flags, cudaEventDisableTiming);
        if (e != cudaSuccess) return fail(nullptr, TRT_ECUDA, cudaGetErrorString(e));
    }
    const int nx = p.nx, G = p.G, M = p.M, N = p.N;
    // host constants
    std::vector<double> hh(nx), mu(M), w(M), Iin0(G, 0.0), IinX(G, 0.0);
    std::vector<double> Ein0(G, 0.0), Fin0(G, 0.0), EinX(G, 0.0), FinX(G, 0.0);
    for (int i = 0; i < nx; ++i) hh[i] = xe[i + 1] - xe[i];
    std::vector<double> ihf(nx + 1, 0.0), hf(nx + 1);
    for (int f = 1; f < nx; ++f) ihf[f] = 1.0 / (hh[f - 1] + hh[f]);
    for (int f = 0; f <= nx; ++f)
        hf[f] = (f == 0) ? 0.5 * hh[0] : (f == nx) ? 0.5 * hh[nx - 1] : 0.5 * (hh[f - 1] + hh[f]);
    std::vector<double> hc(nx), h2(nx), fwl(nx + 1, 0.0), fwr(nx + 1, 0.0);
    for (int i = 0; i < nx; ++i) {
        hc[i] = kC * hh[i];
        h2[i] = 2.0 * hh[i];
    }
    for (int f = 1; f < nx; ++f) {
        fwl[f] = hf[f] * ihf[f] * hh[f - 1];
        fwr[f] = hf[f] * ihf[f] * hh[f];
    }
    std::vector<int> lo_slot(nx + 1, 0);   // chunk layout of the partitioned LO solve
    if (nx >= 2) {
        const int P = std::min(32, nx / 2);
        for (int f = 0; f <= nx; ++f) {
            int l, k;
            if (f == nx) {
                l = P - 1;
                k = nx - ((P - 1) * nx) / P;
            } else {
                l = (f * P) / nx;
                if (l + 1 < P && ((l + 1) * nx) / P <= f) ++l;
                k = f - (l * nx) / P;
            }
            lo_slot[f] = k * 32 + l;
        }
    }
    {
        std::vector<double> x(N), wx(N);
        gauss_legendre_host(N, x.data(), wx.data());
        for (int k = 0; k < N; ++k) {
            mu[k] = 0.5 * (1.0 + x[k]);
            w[k] = 0.5 * wx[k];
            mu[N + k] = -mu[k];
            w[N + k] = w[k];
        }
    }
    if (p.Tl > 0) host_group_B(G, edges.data(), p.Tl, Iin0.data());
    if (p.Tr > 0) host_group_B(G, edges.data(), p.Tr, IinX.data());
    for (int g = 0; g < G; ++g)
        for (int m = 0; m < M; ++m) {
            if (m < N) {
                Ein0[g] += w[m] * Iin0[g] / kC;
                Fin0[g] += w[m] * mu[m] * Iin0[g];
            } else {
                EinX[g] += w[m] * IinX[g] / kC;
                FinX[g] += w[m] * mu[m] * IinX[g];
            }
        }
    // initial state (Sec. 6): T = T0, I = B_g(T0) on every corner and direction
    std::vector<double> B0(G), T0v(nx, p.T0), Eg((size_t)G * nx), Fg((size_t)G * (nx + 1));
    std::vector<double> f((size_t)G * nx), fb(G), C0v(G), CXv(G), Eg0(nx, 0.0), Fg0(nx + 1, 0.0);
    host_group_B(G, edges.data(), p.T0, B0.data());
    for (int g = 0; g < G; ++g) {
        double s0 = 0, s1 = 0, s2 = 0, hm0 = 0, hm1 = 0, hp0 = 0, hp1 = 0;
        for (int m = 0; m < M; ++m) {
            s0 += w[m] * B0[g];
            s1 += w[m] * mu[m] * B0[g];
            s2 += w[m] * mu[m] * mu[m] * B0[g];
            if (m >= N) { hm0 += w[m] * B0[g]; hm1 += w[m] * mu[m] * B0[g]; }
            else { hp0 += w[m] * B0[g]; hp1 += w[m] * mu[m] * B0[g]; }
        }
        double fg = (s0 != 0.0) ? s2 / s0 : 1.0 / 3.0;
        for (int i = 0; i < nx; ++i) {
            Eg[(size_t)g * nx + i] = s0 / kC;
            f[(size_t)g * nx + i] = fg;
            Eg0[i] += s0 / kC;
        }
        for (int i = 0; i <= nx; ++i) {
            Fg[(size_t)g * (nx + 1) + i] = s1;
            Fg0[i] += s1;
        }
        fb[g] = fg;
        C0v[g] = (hm0 != 0.0) ? hm1 / hm0 : -0.5;
        CXv[g] = (hp0 != 0.0) ? hp1 / hp0 : 0.5;
    }
    auto up = [&](double *dst, const std::vector<double> &src) {
        return cudaMemcpyAsync(dst, src.data(), src.size() * sizeof(double),
                               cudaMemcpyHostToDevice, p.stream);
    };
    CK(up(p.h, hh)); CK(up(p.ihf, ihf)); CK(up(p.hf, hf)); CK(up(p.edges, edges)); CK(up(p.mu, mu)); CK(up(p.w, w));
    CK(up(p.hc, hc)); CK(up(p.h2, h2)); CK(up(p.fwl, fwl)); CK(up(p.fwr, fwr));
    CK(cudaMemcpyAsync(p.lo_slot, lo_slot.data(), lo_slot.size() * sizeof(int),
                       cudaMemcpyHostToDevice, p.stream));
    std::vector<float> dir32(4 * (size_t)p.M);   // the FP32 sweeps' per-direction constants
    for (int m = 0; m < p.M; ++m) {
        dir32[4 * m + 0] = (float)std::fabs(mu[m]);
        dir32[4 * m + 1] = (float)(0.5 * std::fabs(mu[m]));
        dir32[4 * m + 2] = (float)(0.5 * w[m]);
        dir32[4 * m + 3] = (float)(0.5 * w[m] * mu[m] * mu[m]);
    }
    CK(cudaMemcpyAsync(p.dir32, dir32.data(), dir32.size() * sizeof(float),
                       cudaMemcpyHostToDevice, p.stream));
    CK(cudaMemcpyAsync(p.e2tab, host_series().e2, 32 * sizeof(double), cudaMemcpyHostToDevice,
                       p.stream));
    CK(up(p.Iin0, Iin0)); CK(up(p.IinX, IinX)); CK(up(p.Ein0, Ein0)); CK(up(p.Fin0, Fin0));
    CK(up(p.EinX, EinX)); CK(up(p.FinX, FinX));
    CK(up(H->T, T0v)); CK(up(H->Eg, Eg)); CK(up(H->Fg, Fg)); CK(up(H->f, f));
    CK(up(H->fb0, fb)); CK(up(H->fbX, fb)); CK(up(H->C0, C0v)); CK(up(H->CX, CXv));
    CK(up(H->grey.E, Eg0)); CK(up(H->grey.F, Fg0));
    CK(up(H->sigE, B0));   // B0 staged for the fill kernel
    const long rows = (long)M * nx * 2;
    const size_t nI = (size_t)rows * p.ldG;
    const int nb = (int)std::min<long>(4096, (long)((nI + 255) / 256));
    if (!sweep_fp32(p.precision)) {
        k_fill_intensity<double><<<nb, 256, 0, p.stream>>>((double *)H->I_cur, H->sigE, rows, p.ldG, G);
        k_fill_intensity<double><<<nb, 256, 0, p.stream>>>((double *)H->I_alt, H->sigE, rows, p.ldG, G);
    } else {
        k_fill_intensity<float><<<nb, 256, 0, p.stream>>>((float *)H->I_cur, H->sigE, rows, p.ldG, G);
        k_fill_intensity<float><<<nb, 256, 0, p.stream>>>((float *)H->I_alt, H->sigE, rows, p.ldG, G);
    }
    CK(cudaGetLastError());
    CK(launch_otab_build(p));   // opacity tables of this group structure
    CK(launch_lo_pair_consts(p));
    CK(cudaMemsetAsync(H->flags, 0, 10 * sizeof(double), p.stream));
    CK(cudaStreamSynchronize(p.stream));
    *out = hp.release();
    return TRT_OK;
}

int trt_destroy(trt_handle *h)
{
    delete h;
    return TRT_OK;
}

const char *trt_last_error(const trt_handle *h)
{
    return h ? h->err.c_str() : g_create_error.c_str();
}

int trt_dims(const trt_handle *h, int *nx, int *N, int *M, int *G, int *ldG, int *n_levels,
             int *precision)
{
    if (!h) return TRT_EINVAL;
    if (nx) *nx = h->p.nx;
    if (N) *N = h->p.N;
    if (M) *M = h->p.M;
    if (G) *G = h->p.G;
    if (ldG) *ldG = h->p.ldG;
    if (n_levels) *n_levels = h->p.nlev;
    if (precision) *precision = h->p.precision;
    return TRT_OK;
}

int trt_step(trt_handle *h, double dt, const trt_cycle *cyc, trt_stats *stats)
{
    if (!h) return TRT_EINVAL;
    if (!cyc || !(dt > 0) || cyc->l_max < 1 || cyc->max_outer < 1 || cyc->type < 0 ||
        cyc->type > 2)
        return fail(h, TRT_EINVAL, "bad step arguments");
    auto t_start = std::chrono::steady_clock::now();
    (void)cudaGetLastError();
    Problem &p = h->p;
    const int nx = p.nx, G = p.G;
    std::vector<int> S;
    schedule(cyc->type, p.nlev, S);
    const int K = (int)S.size();
    const bool fixed = cyc->eps < 0;
    const double eps = cyc->eps, eps_in = cyc->eps_inner;
    int n_ti = 0, n_c = 0, n_lo = 0, s = 0, status = TRT_OK, nk = 0;
    bool swept = false, opac_valid = false;
    int have_prev = 0;
    // the gate is set only around the cycle launches; cleared on every way out
    struct GateOff {
        Problem &p;
        ~GateOff() { p.gate = nullptr; }
    } gate_off{p};
    p.gate = nullptr;

    CK(ensure_lo_consts(p, dt));   // the LO rows' h/dt and hf/(c dt)
    CK(d2d(h, h->Told, h->T, nx));
    CK(d2d(h, h->Eg_old, h->Eg, (size_t)G * nx));
    CK(d2d(h, h->Fg_old, h->Fg, (size_t)G * (nx + 1)));
    CK(launch_group_sum(p, G, h->Eg_old, h->Ephase));
    ++nk;
    // T_r option: the grey energy the opacities read, until the step's first grey solve
    // writes it: the sum of the group energies
    const double *Erad = p.tr_mode ? h->grey.E : nullptr;
    if (p.tr_mode) CK(d2d(h, h->grey.E, h->Ephase, nx));
    CK(cudaMemsetAsync(h->flags, 0, 10 * sizeof(double), p.stream));   // flags and ctl
    if (h->mlp_params) {
        // learned warm start: the s = 0 phase takes f_g from the MLP instead of f_g^{j-1}
        CK(launch_opacity(p, h->T, h->sigE, h->emis, h->sigR, nullptr, nullptr, 0.0, Erad));
        opac_valid = true;
        const int rows = G * nx;
        int rc = trt_mlp_features(nx, G, h->T, h->sigE, h->Eg_old, h->Ephase, h->mlp_x, p.stream);
        if (rc == TRT_OK)
            rc = trt_mlp_forward_fused(rows, h->mlp_x, h->mlp_params, h->mlp_w16, h->mlp_y,
                                       p.stream);
        if (rc != TRT_OK) return fail(h, rc, "closure: MLP inference failed");
        CK(launch_f_from_mlp(p, h->mlp_y, h->f));
        nk += 6;
    }
    Level fine = fine_level(h);
    // LO solves of one cycle: every fine group, the coarse groups of the schedule's grids
    // and one grey solve per visit
    int lo_per_cycle = G + K + 1;
    for (int k = 0; k < K; ++k) lo_per_cycle += p.levels[S[k] - 1];

    bool opac_next = false;   // the phase's opacities already enqueued (below)
    // which source's sums of Eold and Fold (fixed within a step) the grey level holds
    int grey_old = 0;
    for (;;) {
        if (s > 0) {
            if (!opac_next) {
                CK(launch_opacity(p, h->T, h->sigE, h->emis, h->sigR, h->sig32, h->emis32, dt,
                                  Erad));
                ++nk;
            }
            opac_next = false;
            opac_valid = true;
            if (h->sig32)
                CK(launch_sweep(p, dt, h->sig32, h->emis32, true, h->I_cur, h->I_alt, h->part,
                                h->psi_exit, h->f, h->fb0, h->fbX, h->C0, h->CX));
            else
                CK(launch_sweep(p, dt, h->sigE, h->emis, false, h->I_cur, h->I_alt, h->part,
                                h->psi_exit, h->f, h->fb0, h->fbX, h->C0, h->CX));
            nk += 2;
            ++n_ti;
            swept = true;
        }
        // the phase's references (Ephase from the grey E of the phase before) and its gate
        CK(launch_phase_start(h, s > 0));
        ++nk;
        // All l_max cycles are enqueued at once; the cycle kernels return at entry once the
        // cycle before has met the inner test (or found a bad temperature), as decided by
        // its last grey visit on the device, so the host waits once per phase.
        p.gate = h->ctl;
        for (int l = 0; l < cyc->l_max; ++l) {
            if (!opac_valid) {
                CK(launch_opacity(p, h->T, h->sigE, h->emis, h->sigR, nullptr, nullptr, 0.0,
                                  Erad));
                ++nk;
            }
            opac_valid = true;
            CK(launch_lo_solve(p, dt, fine));
            ++nk;
            // grey visit k reads T~^[k] and writes T~^[k+1]: T~^[0] = T, the last visit
            // writes T, the ones between alternate over Ttil and Tnew
            for (int k = 0; k <= K; ++k) {
                double *Tst = (k == 0) ? h->T : (((k - 1) & 1) ? h->Tnew : h->Ttil);
                double *Tout = (k == K) ? h->T : ((k & 1) ? h->Tnew : h->Ttil);
                Level *src = &fine;
                if (k > 0) {
                    const int ng = p.levels[S[k - 1] - 1];
                    CK(launch_opacity(p, Tst, h->sigE, h->emis, h->sigR, nullptr, nullptr, 0.0,
                                      Erad));
                    opac_valid = false;
                    h->crs.n = ng;
                    CK(launch_restrict(p, fine, h->crs));
                    CK(launch_lo_solve(p, dt, h->crs));
                    nk += 3;
                    src = &h->crs;
                }
                GreyArgs a{};
                a.Tstar = Tst; a.Told = h->Told; a.sig_prev = h->sig_prev; a.T_prev = h->T_prev;
                a.T = Tout; a.sig_prev_out = h->sig_prev; a.T_prev_out = h->T_prev;
                a.have_prev = have_prev;
                a.secant_cut = K == 0 ? 0.0 : kSecantCut;   // grey solves on one grid / across grids
                a.cv = p.cv; a.s = p.s; a.dt = dt;
                a.nu_first = p.nu_first; a.nu_last = p.nu_last;
                a.want_norms = (k == K);
                a.Tcyc = h->Tcyc; a.Ecyc = h->Ecyc; a.Tphase = h->Tphase; a.Ephase = h->Ephase;
                a.flags = h->flags;
                if (k == K) {   // the cycle's last visit: end-of-cycle copies, inner-loop control
                    a.Tcyc_out = h->Tcyc; a.Ecyc_out = h->Ecyc;
                    a.ctl = h->ctl; a.eps_in = eps_in; a.fixed = fixed ? 1 : 0;
                }
                // the restriction to the grey level, which forms the visit's per-cell
                // Newton terms too where its two-stage form runs
                const GreyArgs ready = grey_args_ready(p, a);
                bool formed = false;
                CK(launch_restrict(p, *src, h->grey, &ready, h->gpre, &formed, &grey_old));
                a.pre = formed ? h->gpre : nullptr;
                CK(launch_grey(p, h->grey, a));
                nk += 2;   // restriction to grey + grey Newton
                have_prev = 1;
            }
            opac_valid = false;
        }
        p.gate = nullptr;
        CK(cudaMemcpyAsync(h->hflags, h->flags, 10 * sizeof(double), cudaMemcpyDeviceToHost,
                           p.stream));
        CK(cudaEventRecord(h->ev_flags, p.stream));
        // The next phase's opacity evaluation at the phase's final T goes in before the host
        // reads the flags, so that it runs during the round trip.  A step that ends here
        // begins the next one by evaluating the opacities at the same T, so nothing reads
        // these values; the T_r option is left out (the panel loop of its quadrature needs
        // a valid temperature, and a bad one is only known from the flags).
        if (!p.tr_mode && s + 1 < cyc->max_outer) {
            CK(launch_opacity(p, h->T, h->sigE, h->emis, h->sigR, h->sig32, h->emis32, dt, Erad));
            ++nk;
            opac_next = true;
        }
        CK(cudaEventSynchronize(h->ev_flags));
        const double *fl = h->hflags;
        n_c = reinterpret_cast<const int *>(fl + 8)[1];   // cycles run in the step so far
        if (fl[0] != 0.0) {
            status = fail(h, TRT_ENUMERIC, "non-positive or non-finite temperature");
            goto done;
        }
        // the outer test on the phase's last cycle (the flags of the cycles that ran)
        const bool conv_out = fl[5] <= eps * fl[2] && fl[6] <= eps * fl[4];
        ++s;
        if (fixed) {
            if (s >= cyc->max_outer) break;
        } else {
            if (conv_out) break;
            if (s >= cyc->max_outer) {
                status = fail(h, TRT_ENOTCONVERGED, "outer iterations reached max_outer");
                break;
            }
        }
    }
done:
    n_lo = n_c * lo_per_cycle;
    CK(d2d(h, h->Eg, h->E1, (size_t)G * nx));
    CK(d2d(h, h->Fg, h->F1, (size_t)G * (nx + 1)));
    if (swept) std::swap(h->I_cur, h->I_alt);
    CK(cudaStreamSynchronize(p.stream));
    if (stats) {
        stats->n_ti = n_ti; stats->n_c = n_c; stats->n_lo = n_lo; stats->n_outer = s;
        stats->ms = std::chrono::duration<double, std::milli>(std::chrono::steady_clock::now() - t_start).count();
        stats->status = status;
        stats->n_kernels = nk;
    }
    return status;
}

int trt_moments(trt_handle *h, double *T, double *Eg, double *Fg, double *E, double *F)
{
    if (!h) return TRT_EINVAL;
    const Problem &p = h->p;
    const size_t nx = p.nx, G = p.G;
    auto dn = [&](double *dst, const double *src, size_t n) {
        return dst ? cudaMemcpyAsync(dst, src, n * sizeof(double), cudaMemcpyDeviceToHost, p.stream)
                   : cudaSuccess;
    };
    CK(dn(T, h->T, nx));
    CK(dn(Eg, h->Eg, G * nx));
    CK(dn(Fg, h->Fg, G * (nx + 1)));
    CK(dn(E, h->grey.E, nx));
    CK(dn(F, h->grey.F, nx + 1));
    CK(cudaStreamSynchronize(p.stream));
    return TRT_OK;
}

int trt_intensity(trt_handle *h, double *I, double *f)
{
    if (!h) return TRT_EINVAL;
    const Problem &p = h->p;
    const size_t nI = (size_t)p.M * p.nx * 2 * p.ldG;
    if (I) {
        if (!sweep_fp32(p.precision)) {
            CK(cudaMemcpyAsync(I, h->I_cur, nI * sizeof(double), cudaMemcpyDeviceToHost, p.stream));
            CK(cudaStreamSynchronize(p.stream));
        } else {
            std::vector<float> tmp(nI);
            CK(cudaMemcpyAsync(tmp.data(), h->I_cur, nI * sizeof(float), cudaMemcpyDeviceToHost, p.stream));
            CK(cudaStreamSynchronize(p.stream));
            for (size_t k = 0; k < nI; ++k) I[k] = tmp[k];
        }
    }
    if (f) {
        CK(cudaMemcpyAsync(f, h->f, (size_t)p.G * p.nx * sizeof(double), cudaMemcpyDeviceToHost,
                           p.stream));
        CK(cudaStreamSynchronize(p.stream));
    }
    return TRT_OK;
}

int trt_set_state(trt_handle *h, const double *T, const double *Eg, const double *Fg,
                  const double *I, const double *f, const double *fb0, const double *fbX,
                  const double *C0, const double *CX)
{
    if (!h) return TRT_EINVAL;
    const Problem &p = h->p;
    const size_t nx = p.nx, G = p.G;
    auto upd = [&](double *dst, const double *src, size_t n) {
        return src ? cudaMemcpyAsync(dst, src, n * sizeof(double), cudaMemcpyHostToDevice, p.stream)
                   : cudaSuccess;
    };
    CK(upd(h->T, T, nx));
    CK(upd(h->Eg, Eg, G * nx));
    CK(upd(h->Fg, Fg, G * (nx + 1)));
    CK(upd(h->f, f, G * nx));
    CK(upd(h->fb0, fb0, G));
    CK(upd(h->fbX, fbX, G));
    CK(upd(h->C0, C0, G));
    CK(upd(h->CX, CX, G));
    std::vector<float> tmp;
    if (I) {
        const size_t nI = (size_t)p.M * p.nx * 2 * p.ldG;
        if (!sweep_fp32(p.precision)) {
            CK(cudaMemcpyAsync(h->I_cur, I, nI * sizeof(double), cudaMemcpyHostToDevice, p.stream));
        } else {
            tmp.resize(nI);
            for (size_t k = 0; k < nI; ++k) tmp[k] = (float)I[k];
            CK(cudaMemcpyAsync(h->I_cur, tmp.data(), nI * sizeof(float), cudaMemcpyHostToDevice,
                               p.stream));
        }
    }
    if (Eg) CK(launch_group_sum(h->p, (int)G, h->Eg, h->grey.E));
    CK(cudaStreamSynchronize(p.stream));
    return TRT_OK;
}

// ---- kernel-level entry points ----
int trt_k_opacity(trt_handle *h, const double *T, double *sigE, double *emis, double *sigR)
{
    if (!h || !T || !sigE || !emis || !sigR) return TRT_EINVAL;
    CK(launch_opacity(h->p, T, sigE, emis, sigR));
    CK(cudaStreamSynchronize(h->p.stream));
    return TRT_OK;
}

int trt_k_opacity_tr(trt_handle *h, const double *T, const double *Erad, double *sigE,
                     double *emis, double *sigR)
{
    if (!h || !T || !Erad || !sigE || !emis || !sigR || !h->p.tr_mode) return TRT_EINVAL;
    CK(launch_opacity(h->p, T, sigE, emis, sigR, nullptr, nullptr, 0.0, Erad));
    CK(cudaStreamSynchronize(h->p.stream));
    return TRT_OK;
}

int trt_k_sweep(trt_handle *h, double dt, const double *sigE, const double *emis,
                const void *I_old, void *I_new, double *f, double *fb0, double *fbX,
                double *C0, double *CX)
{
    if (!h || !(dt > 0) || !sigE || !emis || !I_old || !I_new || !f || !fb0 || !fbX || !C0 || !CX)
        return TRT_EINVAL;
    if (h->sig32) {   // FP32 sweeps: the step's pre-scaled FP32 inputs, as a step forms them
        CK(launch_prescale32(h->p, dt, sigE, emis, h->sig32, h->emis32));
        CK(launch_sweep(h->p, dt, h->sig32, h->emis32, true, I_old, I_new, h->part, h->psi_exit,
                        f, fb0, fbX, C0, CX));
    } else {
        CK(launch_sweep(h->p, dt, sigE, emis, false, I_old, I_new, h->part, h->psi_exit, f, fb0,
                        fbX, C0, CX));
    }
    CK(cudaStreamSynchronize(h->p.stream));
    return TRT_OK;
}

int trt_set_closure(trt_handle *h, const float *params, const void *w16, void *scratch,
                    size_t scratch_bytes, float *x, float *y)
{
    if (!h) return TRT_EINVAL;
    if (!params) {
        h->mlp_params = nullptr;
        return TRT_OK;
    }
    const int rows = h->p.G * h->p.nx;
    if (!w16 || !scratch || !x || !y || scratch_bytes < trt_mlp_scratch_bytes(rows, 0))
        return fail(h, TRT_EINVAL, "trt_set_closure: missing buffer or scratch too small");
    if (reinterpret_cast<uintptr_t>(params) & 15)
        return fail(h, TRT_EINVAL, "trt_set_closure: params not 16-byte aligned");
    h->mlp_params = params;
    h->mlp_w16 = w16;
    h->mlp_scratch = scratch;
    h->mlp_scratch_bytes = scratch_bytes;
    h->mlp_x = x;
    h->mlp_y = y;
    return TRT_OK;
}

int trt_fp64_peak(int reps, void *stream, double *tflops)
{
    if (reps < 1 || !tflops) return TRT_EINVAL;
    float ms = 0.f;
    long long fmas = 0;
    if (fp64_probe(reps, reinterpret_cast<cudaStream_t>(stream), &ms, &fmas) != cudaSuccess ||
        !(ms > 0.f))
        return TRT_ECUDA;
    *tflops = 2.0 * (double)fmas / (ms * 1e-3) / 1e12;
    return TRT_OK;
}

int trt_k_fastmath(int n, const double *x, double *ex, double *rc, void *stream)
{
    if (n < 1 || !x || !ex || !rc) return TRT_EINVAL;
    return launch_fastmath(n, x, ex, rc, reinterpret_cast<cudaStream_t>(stream)) == cudaSuccess
               ? TRT_OK
               : TRT_ECUDA;
}

int trt_sweep_shapes(const trt_handle *h)
{
    return h ? sweep_shape_count(h->p.precision) : 0;
}

int trt_set_sweep_tile(trt_handle *h, int D, int shape)
{
    if (!h) return TRT_EINVAL;
    int cand[3];
    const int nc = sweep_D_candidates(h->p, cand);
    bool ok = false;
    for (int i = 0; i < nc; ++i) ok = ok || cand[i] == D;
    if (!ok || !sweep_tile_ok(h->p.precision, D, shape))
        return fail(h, TRT_EINVAL, "trt_set_sweep_tile: D or shape not a candidate");
    h->p.sweep_D = D;
    h->p.sweep_shape = shape;
    return TRT_OK;
}

int trt_get_sweep_tile(const trt_handle *h, int *D, int *shape)
{
    if (!h) return TRT_EINVAL;
    if (D) *D = h->p.sweep_D;
    if (shape) *shape = h->p.sweep_shape;
    return TRT_OK;
}

int trt_sweep_time(trt_handle *h, double dt, int reps, float *ms)
{
    if (!h || !(dt > 0) || reps < 1 || !ms) return TRT_EINVAL;
    const Problem &p = h->p;
    if (p.nx < 3) return fail(h, TRT_EINVAL, "trt_sweep_time needs n_cells >= 3");
    // outputs go to scratch that no step reads before writing it: the fine-solve arrays
    // E1 [G][nx] (f) and F1 [G][nx+1] (the four boundary arrays, 4 G <= G (nx + 1))
    double *f = h->E1, *b = h->F1;
    const size_t G = p.G;
    CK(launch_opacity(p, h->T, h->sigE, h->emis, h->sigR, h->sig32, h->emis32, dt));
    auto one = [&]() {
        return h->sig32 ? launch_sweep(p, dt, h->sig32, h->emis32, true, h->I_cur, h->I_alt,
                                       h->part, h->psi_exit, f, b, b + G, b + 2 * G, b + 3 * G)
                        : launch_sweep(p, dt, h->sigE, h->emis, false, h->I_cur, h->I_alt,
                                       h->part, h->psi_exit, f, b, b + G, b + 2 * G, b + 3 * G);
    };
    CK(one());
    cudaEvent_t e0, e1;
    CK(cudaEventCreate(&e0));
    CK(cudaEventCreate(&e1));
    cudaError_t e = cudaEventRecord(e0, p.stream);
    for (int r = 0; r < reps && e == cudaSuccess; ++r) e = one();
    if (e == cudaSuccess) e = cudaEventRecord(e1, p.stream);
    if (e == cudaSuccess) e = cudaEventSynchronize(e1);
    float t = 0;
    if (e == cudaSuccess) e = cudaEventElapsedTime(&t, e0, e1);
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    CK(e);
    *ms = t / reps;
    return TRT_OK;
}

int trt_autotune(trt_handle *h, double dt, int reps, int *D, int *S, int *NS)
{
    if (!h || !(dt > 0) || reps < 1) return TRT_EINVAL;
    int cand[3];
    const int nc = sweep_D_candidates(h->p, cand);
    const int ns = sweep_shape_count(h->p.precision);
    const int D0 = h->p.sweep_D, sh0 = h->p.sweep_shape;
    float best = 1e30f;
    int bD = D0, bsh = sh0;
    for (int i = 0; i < nc; ++i) {
        for (int k = 0; k < ns; ++k) {
            if (!sweep_tile_ok(h->p.precision, cand[i], k)) continue;
            h->p.sweep_D = cand[i];
            h->p.sweep_shape = k;
            float ms = 0;
            const int rc = trt_sweep_time(h, dt, reps, &ms);
            if (rc == TRT_ECUDA) {
                // a shape the device cannot launch (shared memory) is skipped; a sticky
                // error is not
                cudaGetLastError();
                if (cudaStreamSynchronize(h->p.stream) != cudaSuccess) {
                    h->p.sweep_D = D0;
                    h->p.sweep_shape = sh0;
                    return TRT_ECUDA;
                }
                continue;
            }
            if (rc != TRT_OK) {
                h->p.sweep_D = D0;
                h->p.sweep_shape = sh0;
                return rc;
            }
            if (ms < best) {
                best = ms;
                bD = cand[i];
                bsh = k;
            }
        }
    }
    h->p.sweep_D = bD;
    h->p.sweep_shape = bsh;
    int s_ = 0, ns_ = 0;
    sweep_shape_info(h->p.precision, bsh, &s_, &ns_);
    if (D) *D = bD > 0 ? bD : cand[0];
    if (S) *S = s_;
    if (NS) *NS = ns_;
    return TRT_OK;
}

int trt_level_view(trt_handle *h, int which, trt_level *out)
{
    if (!h || !out || which < 0 || which > 2) return TRT_EINVAL;
    const Level L = which == 0 ? fine_level(h) : which == 1 ? h->crs : h->grey;
    out->n = L.n; out->fine = L.fine;
    out->phi = L.phi; out->sig = L.sig; out->emis = L.emis; out->Eold = L.Eold;
    out->Esum = L.Esum; out->sigR = L.sigR; out->etaR = L.etaR; out->etaL = L.etaL;
    out->Fold = L.Fold; out->phib0 = L.phib0; out->phibX = L.phibX; out->C0 = L.C0;
    out->CX = L.CX; out->Ein0 = L.Ein0; out->Fin0 = L.Fin0; out->EinX = L.EinX;
    out->FinX = L.FinX; out->E = L.E; out->F = L.F; out->Eb0 = L.Eb0; out->EbX = L.EbX;
    return TRT_OK;
}

int trt_k_lo_solve(trt_handle *h, double dt, trt_level *lv)
{
    if (!h || !lv || !(dt > 0) || lv->n < 1) return TRT_EINVAL;
    Level L = from_abi(lv);
    CK(ensure_lo_consts(h->p, dt));
    CK(launch_lo_solve(h->p, dt, L));
    CK(cudaStreamSynchronize(h->p.stream));
    return TRT_OK;
}

int trt_k_restrict(trt_handle *h, const trt_level *src, trt_level *dst)
{
    if (!h || !src || !dst || dst->n < 1 || src->n < dst->n || src->n % dst->n) return TRT_EINVAL;
    if (dst->n > 65535) return TRT_EINVAL;
    Level S = from_abi(src), T = from_abi(dst);
    CK(launch_restrict(h->p, S, T));
    CK(cudaStreamSynchronize(h->p.stream));
    return TRT_OK;
}

int trt_k_grey_newton(trt_handle *h, double dt, const double *Tstar, const double *Told,
                      const double *sig_prev, const double *T_prev, int have_prev,
                      double secant_cut, trt_level *g, double *T)
{
    if (!h || !g || g->n != 1 || !(dt > 0) || !Tstar || !Told || !T) return TRT_EINVAL;
    if (have_prev && (!sig_prev || !T_prev)) return TRT_EINVAL;
    Level L = from_abi(g);
    CK(ensure_lo_consts(h->p, dt));
    const Problem &p = h->p;
    GreyArgs a{};
    a.Tstar = Tstar; a.Told = Told;
    a.sig_prev = have_prev ? sig_prev : Tstar;
    a.T_prev = have_prev ? T_prev : Tstar;
    a.T = T;
    a.sig_prev_out = h->part;             // scratch, not state
    a.T_prev_out = h->part + p.nx;
    a.have_prev = have_prev;
    a.secant_cut = secant_cut;
    a.cv = p.cv; a.s = p.s; a.dt = dt;
    a.nu_first = p.nu_first; a.nu_last = p.nu_last;
    a.want_norms = 0;
    a.Tcyc = a.Ecyc = a.Tphase = a.Ephase = nullptr;
    a.flags = h->flags;
    CK(cudaMemsetAsync(h->flags, 0, 8 * sizeof(double), p.stream));
    CK(launch_grey(p, L, a));
    CK(cudaMemcpyAsync(h->hflags, h->flags, 8 * sizeof(double), cudaMemcpyDeviceToHost, p.stream));
    CK(cudaStreamSynchronize(p.stream));
    if (h->hflags[0] != 0.0) return fail(h, TRT_ENUMERIC, "non-positive or non-finite temperature");
    return TRT_OK;
}

}  // extern "C"
