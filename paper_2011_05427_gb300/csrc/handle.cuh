// handle.cuh -- the solver handle of include/trt.h and helpers shared by the single-slab
// driver (api.cu) and the batched driver (batch.cu).
#pragma once
#include <string>
#include <vector>
#include "common.cuh"

struct trt_handle {
    trt::Problem p;
    double *T, *Told, *Tcyc, *Tphase, *Ttil, *Tnew, *sig_prev, *T_prev;
    double *Eg, *Fg, *Eg_old, *Fg_old;
    void *I_cur, *I_alt;
    double *f, *fb0, *fbX, *C0, *CX;
    double *sigE, *emis, *sigR;
    float *sig32 = nullptr, *emis32 = nullptr;   // FP32 copies for an FP32 sweep
    double *part, *psi_exit;
    double *E1, *F1, *Eb0_1, *EbX_1;
    double *gpre;   // [3][nx]: the grey Newton terms formed by the restriction
    trt::Level crs, grey;
    double *Ecyc, *Ephase;
    double *flags = nullptr;    // [10]: convergence flags [0..6], then the inner-loop
    int *ctl = nullptr;         // control words (ints in the last two doubles of flags)
    double *hflags = nullptr;   // pinned host mirror of flags + ctl, owned (freed below)
    cudaEvent_t ev_flags = nullptr;   // recorded after each phase's flags copy, owned
    // learned closure (trt_set_closure): caller-owned device buffers, or null
    const float *mlp_params = nullptr;
    const void *mlp_w16 = nullptr;
    void *mlp_scratch = nullptr;
    size_t mlp_scratch_bytes = 0;
    float *mlp_x = nullptr, *mlp_y = nullptr;
    std::string err;
    ~trt_handle()
    {
        if (hflags) cudaFreeHost(hflags);
        if (ev_flags) cudaEventDestroy(ev_flags);
    }
};

// cycle schedule S of Sec. 4 (grid indices 2..Gamma-1 visited between grey solves)
inline void schedule(int type, int Gamma, std::vector<int> &S)
{
    S.clear();
    if (Gamma <= 2 || type == TRT_CYCLE_V) return;
    if (type == TRT_CYCLE_F) {
        for (int g = Gamma - 1; g >= 2; --g) S.push_back(g);
        return;
    }
    // W: w(Gamma-1) = [Gamma-1]; w(g) = w(g+1) + [g] + w(g+1)
    std::vector<int> cur{Gamma - 1};
    for (int g = Gamma - 2; g >= 2; --g) {
        std::vector<int> nxt(cur);
        nxt.push_back(g);
        nxt.insert(nxt.end(), cur.begin(), cur.end());
        cur.swap(nxt);
    }
    S = cur;
}

inline trt::Level fine_level(trt_handle *h)
{
    trt::Level L;
    L.n = h->p.G;
    L.fine = 1;
    L.phi = h->f; L.sig = h->sigE; L.emis = h->emis; L.Eold = h->Eg_old; L.Esum = nullptr;
    L.sigR = h->sigR; L.etaR = nullptr; L.etaL = nullptr; L.Fold = h->Fg_old;
    L.phib0 = h->fb0; L.phibX = h->fbX; L.C0 = h->C0; L.CX = h->CX;
    L.Ein0 = h->p.Ein0; L.Fin0 = h->p.Fin0; L.EinX = h->p.EinX; L.FinX = h->p.FinX;
    L.E = h->E1; L.F = h->F1; L.Eb0 = h->Eb0_1; L.EbX = h->EbX_1;
    return L;
}

