// batch.cu -- many independent slabs stepped together: Algorithm 3 (Sec. 4) per slab, in
// lockstep, with every kernel launch covering all slabs that take part in it.
//
// Each slab is an ordinary handle carved from its own slice of the caller's workspace.  A
// time step is a sequence of stages (step start, sweep, phase start, cycle, phase end,
// step end); a stage is a fixed list of ops, an op is one batched kernel (batch.cuh) over
// the slabs eligible for it.  Eligibility has a static part, fixed at creation (the
// op's per-slab block counts: zero when the op does not apply to the slab, e.g. a coarse
// visit beyond the slab's schedule or a restriction variant the slab does not use), and a
// dynamic part, one byte per (class, slab) written by the host before the stage runs
// (which slabs sweep now, which are still inside the cycle loop, which need opacities).
// A planner kernel turns both into the ops' work lists on the device, so the argument
// blocks (rebuilt once per step) and the launch sequence are the same for every run of a
// stage: the stage is captured once into a CUDA graph and replayed.  The host reads all
// slabs' convergence flags once per cycle.
//
// Readings and arithmetic are those of the single-slab driver (api.cu); a slab stepped in a
// batch goes through the same kernels on the same data in the same order.
#include <algorithm>
#include <cstring>
#include <memory>
#include <string>
#include <vector>
#include "batch.cuh"
#include "handle.cuh"

using namespace trt;

namespace {

enum Cls { C_ALL = 0, C_SWEEP, C_PHASE, C_CYCLE, C_OPAC0, C_PHASE_END, NCLS };
enum Kind { K_OPAC, K_SWEEP, K_FINAL, K_LO, K_RESTRICT, K_RPART, K_RFINAL, K_GREY, K_GSUM, K_COPY };
enum StageId { S_STEP_START, S_SWEEP, S_PHASE, S_PHASE_END, S_STEP_END, S_CYCLE0 };

struct Op {
    Kind kind;
    int cls;
    int KS = 1;             // K_RESTRICT row slices
    size_t csz = 0;         // bytes of one argument block
    size_t ctx_off = 0;     // byte offset of xs[n] in the argument region
    size_t meta_off = 0;    // int offset of the work list in the meta region
    size_t tab_off = 0;     // int offset of blocks[n], gx[n] in the table region
    std::vector<int> blocks, gx;
    int grid = 0;
    // per slab argument block, rebuilt every step: (slab, dt) -> bytes
    std::vector<unsigned char> host;   // n * csz
};

struct Stage {
    std::vector<Op> ops;
    size_t plan_off = 0;    // offset (PlanOp units) of this stage's planner table
    bool d2h_flags = false;
    cudaGraphExec_t exec = nullptr;
    bool graph_failed = false;
    int cycle_type = -1;
};

struct PlanOp {
    int *meta;
    const int *blocks, *gx;
    int cls;
};

// one block per op: thread 0 lists the eligible slabs of the op's class in slab order
__global__ void k_plan(const PlanOp *__restrict__ ops, int nops, const unsigned char *dyn, int n)
{
    const int o = blockIdx.x;
    if (o >= nops || threadIdx.x != 0) return;
    const PlanOp op = ops[o];
    int *pre = op.meta + 1, *gx = op.meta + 2 + n, *sid = op.meta + 2 + 2 * n;
    int np = 0;
    pre[0] = 0;
    for (int s = 0; s < n; ++s) {
        if (op.blocks[s] > 0 && dyn[op.cls * n + s]) {
            sid[np] = s;
            gx[np] = op.gx[s];
            pre[np + 1] = pre[np] + op.blocks[s];
            ++np;
        }
    }
    op.meta[0] = np;
}

struct SlabState {
    int s = 0, status = TRT_OK, n_ti = 0, n_c = 0, n_lo = 0;
    bool opac_valid = false, swept = false, active = false, conv_out = false, in_cycle = false;
};

}  // namespace

struct trt_batch {
    int n = 0, precision = 0, D = 1, shape = 0, max_nx = 1;
    cudaStream_t st = nullptr;
    std::vector<trt_handle *> h;
    std::vector<int> K;                       // per slab: levels, for schedules
    // device regions (carved from the batch's workspace slice) and pinned mirrors
    unsigned char *d_ctx = nullptr, *h_ctx = nullptr;
    size_t ctx_bytes = 0;
    int *d_meta = nullptr;
    size_t meta_ints = 0;
    int *d_tab = nullptr;
    size_t tab_ints = 0;
    PlanOp *d_plan = nullptr;
    size_t plan_cap = 0;
    unsigned char *d_dyn = nullptr, *h_dyn = nullptr;
    double *d_flags = nullptr, *h_flags = nullptr;
    int *d_have_prev = nullptr;
    Stage stage[S_CYCLE0 + 3];                // + one cycle stage per cycle type
    bool built = false;
    double built_dt = -1.0;
    long layout_key = -1;
    std::string err;
    ~trt_batch()
    {
        for (auto &sg : stage)
            if (sg.exec) cudaGraphExecDestroy(sg.exec);
        for (auto *x : h) trt_destroy(x);
        if (h_ctx) cudaFreeHost(h_ctx);
        if (h_dyn) cudaFreeHost(h_dyn);
        if (h_flags) cudaFreeHost(h_flags);
    }
};

namespace {

int bfail(trt_batch *b, int code, const std::string &msg)
{
    b->err = msg;
    return code;
}

#define BCK(call)                                                                           \
    do {                                                                                    \
        cudaError_t e__ = (call);                                                           \
        if (e__ != cudaSuccess)                                                             \
            return bfail(b, TRT_ECUDA, std::string(#call) + ": " + cudaGetErrorString(e__)); \
    } while (0)

size_t ctx_size(Kind k)
{
    switch (k) {
    case K_OPAC: return sizeof(OpacityArgs);
    case K_SWEEP: return sizeof(SweepArgs);
    case K_FINAL: return sizeof(FinalizeArgs);
    case K_LO: return sizeof(LoCtx);
    case K_RESTRICT: return sizeof(RestrictCtx);
    case K_RPART:
    case K_RFINAL: return sizeof(Restrict2Ctx);
    case K_GREY: return sizeof(GreyCtx);
    case K_GSUM: return sizeof(GroupSumArgs);
    case K_COPY: return sizeof(CopyArgs);
    }
    return 0;
}

int grid_cap(Kind k) { return k == K_SWEEP ? 152 * 2 : 152 * 16; }

// ops of all stages built for one cycle type: the W cycle is the longest (2^(Gamma-2) - 1
// coarse visits); per visit at most opacity + 7 restriction variants + solve + grey
size_t max_ops(int nlev_max)
{
    const size_t K = ((size_t)1 << (std::min(nlev_max, 12) - 2)) - 1;
    return 32 + 18 * (K + 1);
}

// ---- op builders: each knows, per slab, its block count and its argument block ----
struct Builder {
    trt_batch *b;
    double dt;
    const trt_cycle *cyc;   // cycle stages only
    std::vector<std::vector<int>> S;   // schedules per slab (cycle stages)
    Stage *sg;

    Op &add(Kind k, int cls)
    {
        sg->ops.emplace_back();
        Op &o = sg->ops.back();
        o.kind = k;
        o.cls = cls;
        o.csz = ctx_size(k);
        o.blocks.assign(b->n, 0);
        o.gx.assign(b->n, 1);
        o.host.assign((size_t)b->n * o.csz, 0);
        return o;
    }
    template <class T>
    void set(Op &o, int s, const T &x, int blocks, int gx)
    {
        std::memcpy(o.host.data() + (size_t)s * o.csz, &x, sizeof(T));
        o.blocks[s] = blocks;
        o.gx[s] = gx;
    }
    void copy(int cls, const std::vector<CopyArgs> &c)   // one copy per slab (n == 0: none)
    {
        Op &o = add(K_COPY, cls);
        for (int s = 0; s < b->n; ++s)
            if (c[s].n > 0) set(o, s, c[s], (int)((c[s].n + 255) / 256), (int)((c[s].n + 255) / 256));
    }
};

int face_blocks(const Problem &p) { return (p.nx + 1 + 31) / 32; }

}  // namespace

namespace {

// Build every op of stage `id` (cycle stages: for cycle type cyc->type) with its argument
// blocks for time step dt.
void build_stage(trt_batch *b, int id, double dt, int cycle_type)
{
    Stage &sg = b->stage[id];
    sg.ops.clear();
    sg.d2h_flags = false;
    Builder B{b, dt, nullptr, {}, &sg};
    const int n = b->n;
    std::vector<CopyArgs> cp(n);
    auto zero_cp = [&]() { for (auto &c : cp) c = CopyArgs{nullptr, nullptr, 0}; };
    auto H = [&](int s) { return b->h[s]; };

    if (id == S_STEP_START) {
        zero_cp();
        for (int s = 0; s < n; ++s) cp[s] = CopyArgs{H(s)->Told, H(s)->T, H(s)->p.nx};
        B.copy(C_ALL, cp);
        for (int s = 0; s < n; ++s)
            cp[s] = CopyArgs{H(s)->Eg_old, H(s)->Eg, (long)H(s)->p.G * H(s)->p.nx};
        B.copy(C_ALL, cp);
        for (int s = 0; s < n; ++s)
            cp[s] = CopyArgs{H(s)->Fg_old, H(s)->Fg, (long)H(s)->p.G * (H(s)->p.nx + 1)};
        B.copy(C_ALL, cp);
        Op &o = B.add(K_GSUM, C_ALL);
        for (int s = 0; s < n; ++s) {
            GroupSumArgs a{H(s)->p.G, H(s)->p.nx, H(s)->Eg_old, H(s)->Ephase};
            const int nb = (H(s)->p.nx + 31) / 32;
            B.set(o, s, a, nb, nb);
        }
    } else if (id == S_SWEEP) {
        Op &oo = B.add(K_OPAC, C_SWEEP);
        for (int s = 0; s < n; ++s) {
            const Problem &p = H(s)->p;
            B.set(oo, s, make_opacity_args(p, H(s)->T, H(s)->sigE, H(s)->emis, H(s)->sigR,
                                           H(s)->sig32, H(s)->emis32, dt),
                  opacity_blocks(p), opacity_gx(p));
        }
        const size_t isw = sg.ops.size();
        B.add(K_SWEEP, C_SWEEP);
        B.add(K_FINAL, C_SWEEP);
        for (int s = 0; s < n; ++s) {
            trt_handle *x = H(s);
            Problem p = x->p;
            const void *sg_ = x->sig32 ? (const void *)x->sig32 : (const void *)x->sigE;
            const void *em_ = x->sig32 ? (const void *)x->emis32 : (const void *)x->emis;
            SweepArgs a = make_sweep_args(p, dt, sg_, em_, x->I_cur, x->I_alt, x->part,
                                          x->psi_exit, x->f, x->fb0, x->fbX, x->C0, x->CX, b->D);
            if (x->sig32) a.kap32 = x->emis32 + (size_t)p.G * p.nx;   // after e (opacity)
            const int ntile = p.M / b->D;
            B.set(sg.ops[isw], s, a, ntile * sweep_group_tiles(b->precision, b->shape, b->D, p.ldG),
                  ntile);
            p.sweep_D = b->D;
            const FinalizeArgs fa = make_finalize_args(p, a);
            B.set(sg.ops[isw + 1], s, fa, finalize_blocks(p), finalize_blocks(p));
        }
    } else if (id == S_PHASE) {
        zero_cp();
        for (int s = 0; s < n; ++s) cp[s] = CopyArgs{H(s)->Tphase, H(s)->T, H(s)->p.nx};
        B.copy(C_PHASE, cp);
        for (int s = 0; s < n; ++s) cp[s] = CopyArgs{H(s)->Tcyc, H(s)->T, H(s)->p.nx};
        B.copy(C_PHASE, cp);
        for (int s = 0; s < n; ++s) cp[s] = CopyArgs{H(s)->Ecyc, H(s)->Ephase, H(s)->p.nx};
        B.copy(C_PHASE, cp);
    } else if (id == S_PHASE_END) {
        for (int s = 0; s < n; ++s) cp[s] = CopyArgs{H(s)->Ephase, H(s)->grey.E, H(s)->p.nx};
        B.copy(C_PHASE_END, cp);
    } else if (id == S_STEP_END) {
        for (int s = 0; s < n; ++s)
            cp[s] = CopyArgs{H(s)->Eg, H(s)->E1, (long)H(s)->p.G * H(s)->p.nx};
        B.copy(C_ALL, cp);
        for (int s = 0; s < n; ++s)
            cp[s] = CopyArgs{H(s)->Fg, H(s)->F1, (long)H(s)->p.G * (H(s)->p.nx + 1)};
        B.copy(C_ALL, cp);
    } else {
        // one cycle (Algorithm 3 inner loop body) for cycle type `cycle_type`
        sg.d2h_flags = true;
        sg.cycle_type = cycle_type;
        std::vector<std::vector<int>> S(n);
        int Kmax = 0;
        for (int s = 0; s < n; ++s) {
            schedule(cycle_type, H(s)->p.nlev, S[s]);
            Kmax = std::max(Kmax, (int)S[s].size());
        }
        std::vector<Level> fine(n), grey(n), crs(n);
        for (int s = 0; s < n; ++s) {
            fine[s] = fine_level(H(s));
            grey[s] = H(s)->grey;
        }
        auto Tbuf = [&](int s, int k) { return (k & 1) ? H(s)->Tnew : H(s)->Ttil; };
        Op &o0 = B.add(K_OPAC, C_OPAC0);
        for (int s = 0; s < n; ++s) {
            const Problem &p = H(s)->p;
            B.set(o0, s, make_opacity_args(p, H(s)->T, H(s)->sigE, H(s)->emis, H(s)->sigR,
                                           nullptr, nullptr, 0.0),
                  opacity_blocks(p), opacity_gx(p));
        }
        {
            Op &o = B.add(K_LO, C_CYCLE);
            for (int s = 0; s < n; ++s)
                B.set(o, s, make_lo_ctx(H(s)->p, dt, fine[s]), fine[s].n, fine[s].n);
        }
        for (int s = 0; s < n; ++s) cp[s] = CopyArgs{Tbuf(s, 0), H(s)->T, H(s)->p.nx};
        B.copy(C_CYCLE, cp);
        auto restrict_op = [&](const std::vector<Level> &src, const std::vector<Level> &dst,
                               const std::vector<int> &use) {
            // variants: two-stage (part + final), or single with KS in {1, 2, 4, 8, 16}
            int ip = -1, iv[5] = {-1, -1, -1, -1, -1};
            for (int s = 0; s < n; ++s) {
                if (!use[s]) continue;
                const Problem &p = H(s)->p;
                int KS = 1;
                if (restrict_kind(p, src[s].n, dst[s].n, &KS) == 2) {
                    if (ip < 0) {
                        ip = (int)sg.ops.size();
                        B.add(K_RPART, C_CYCLE);
                        B.add(K_RFINAL, C_CYCLE);
                    }
                    const Restrict2Ctx y = make_restrict2_ctx(p, src[s], dst[s]);
                    const int gxx = face_blocks(p);
                    B.set(sg.ops[ip], s, y, gxx * dst[s].n * y.nchunk, gxx);
                    B.set(sg.ops[ip + 1], s, y, gxx * dst[s].n, gxx);
                } else {
                    int idx = 0;
                    while ((1 << idx) < KS) ++idx;
                    if (iv[idx] < 0) {
                        iv[idx] = (int)sg.ops.size();
                        B.add(K_RESTRICT, C_CYCLE).KS = KS;
                    }
                    const int gxx = face_blocks(p);
                    B.set(sg.ops[iv[idx]], s, make_restrict_ctx(p, src[s], dst[s]),
                          gxx * dst[s].n, gxx);
                }
            }
        };
        for (int k = 0; k <= Kmax; ++k) {
            std::vector<int> use(n, 0);
            for (int s = 0; s < n; ++s) use[s] = k <= (int)S[s].size();
            std::vector<Level> src(n);
            if (k > 0) {
                Op &oo = B.add(K_OPAC, C_CYCLE);
                for (int s = 0; s < n; ++s) {
                    if (!use[s]) continue;
                    const Problem &p = H(s)->p;
                    B.set(oo, s, make_opacity_args(p, Tbuf(s, k), H(s)->sigE, H(s)->emis,
                                                   H(s)->sigR, nullptr, nullptr, 0.0),
                          opacity_blocks(p), opacity_gx(p));
                }
                for (int s = 0; s < n; ++s) {
                    crs[s] = H(s)->crs;
                    if (use[s]) crs[s].n = H(s)->p.levels[S[s][k - 1] - 1];
                }
                restrict_op(fine, crs, use);
                Op &ol = B.add(K_LO, C_CYCLE);
                for (int s = 0; s < n; ++s)
                    if (use[s]) B.set(ol, s, make_lo_ctx(H(s)->p, dt, crs[s]), crs[s].n, crs[s].n);
                src = crs;
            } else {
                src = fine;
            }
            restrict_op(src, grey, use);
            Op &og = B.add(K_GREY, C_CYCLE);
            for (int s = 0; s < n; ++s) {
                if (!use[s]) continue;
                trt_handle *x = H(s);
                const Problem &p = x->p;
                GreyArgs a{};
                a.Tstar = Tbuf(s, k); a.T = Tbuf(s, k + 1);
                a.Told = x->Told; a.sig_prev = x->sig_prev; a.T_prev = x->T_prev;
                a.sig_prev_out = x->sig_prev; a.T_prev_out = x->T_prev;
                a.have_prev = 0;
                a.have_prev_dev = b->d_have_prev + s;
                a.secant_cut = S[s].empty() ? 0.0 : kSecantCut;
                a.cv = p.cv; a.s = p.s; a.dt = dt;
                a.nu_first = p.nu_first; a.nu_last = p.nu_last;
                a.want_norms = (k == (int)S[s].size());
                a.Tcyc = x->Tcyc; a.Ecyc = x->Ecyc; a.Tphase = x->Tphase; a.Ephase = x->Ephase;
                a.flags = b->d_flags + 8 * (size_t)s;
                if (a.want_norms) {   // the end-of-cycle copies T, Tcyc = T, Ecyc = grey E
                    a.T_out = x->T; a.Tcyc_out = x->Tcyc; a.Ecyc_out = x->Ecyc;
                }
                B.set(og, s, make_grey_ctx(p, x->grey, a), 1, 1);
            }
        }
    }
    // drop ops nobody is eligible for; fixed grids
    std::vector<Op> keep;
    for (auto &o : sg.ops) {
        long tot = 0;
        for (int v : o.blocks) tot += v;
        if (tot == 0) continue;
        o.grid = (int)std::min<long>(tot, grid_cap(o.kind));
        keep.push_back(std::move(o));
    }
    sg.ops.swap(keep);
}

}  // namespace

extern "C" {

size_t trt_batch_workspace_bytes(int n, const trt_grid *grids, const trt_angles *angles,
                                 const trt_groups *groups, const trt_options *opt)
{
    if (n < 1 || !grids || !angles || !groups || !opt) return 0;
    size_t tot = 0;
    int nlev_max = 2, nx_max = 1;
    for (int s = 0; s < n; ++s) {
        const size_t w = trt_workspace_bytes(&grids[s], &angles[s], &groups[s], opt);
        if (w == 0) return 0;
        tot += (w + 255) / 256 * 256;
        nlev_max = std::max(nlev_max, groups[s].n_levels);
        nx_max = std::max(nx_max, grids[s].n_cells);
    }
    (void)nx_max;
    const size_t mo = max_ops(nlev_max);
    const size_t per_op = (size_t)n * 512 + 256;   // largest argument block < 512 bytes
    tot += mo * per_op;
    tot += mo * (bmeta_ints(n) + n + 64) * sizeof(int);
    tot += mo * (2 * (size_t)n + 64) * sizeof(int);
    tot += mo * sizeof(PlanOp) + 256;
    tot += NCLS * (size_t)n + 256 + 8 * sizeof(double) * (size_t)n + 256 + sizeof(int) * n + 256;
    return tot + 4096;
}

int trt_create_batch(int n, const trt_grid *grids, const trt_angles *angles,
                     const trt_groups *groups, const trt_opacity *opacities, const double *cv,
                     const trt_options *opt, trt_batch **out)
{
    if (out) *out = nullptr;
    if (n < 1 || !grids || !angles || !groups || !opacities || !cv || !opt || !out)
        return TRT_EINVAL;
    const size_t need = trt_batch_workspace_bytes(n, grids, angles, groups, opt);
    if (need == 0) return TRT_EINVAL;
    if (!opt->workspace || opt->workspace_bytes < need) return TRT_ENOSPACE;
    std::unique_ptr<trt_batch> B(new trt_batch());
    trt_batch *b = B.get();
    b->n = n;
    b->precision = opt->precision;
    b->st = reinterpret_cast<cudaStream_t>(opt->stream);
    char *base = reinterpret_cast<char *>(opt->workspace);
    size_t off = 0;
    for (int s = 0; s < n; ++s)   // the T_r option is single-slab only
        if (opacities[s].tr_mode) return TRT_EINVAL;
    for (int s = 0; s < n; ++s) {
        trt_options o = *opt;
        const size_t w = trt_workspace_bytes(&grids[s], &angles[s], &groups[s], opt);
        o.workspace = base + off;
        o.workspace_bytes = w;
        trt_handle *x = nullptr;
        const int rc = trt_create(&grids[s], &angles[s], &groups[s], &opacities[s], cv[s], &o, &x);
        if (rc != TRT_OK) return rc;
        b->h.push_back(x);
        off += (w + 255) / 256 * 256;
        b->max_nx = std::max(b->max_nx, grids[s].n_cells);
    }
    // directions per CTA of the batched sweep: one D for every slab (a divisor of every N,
    // and no smaller than any slab's smallest candidate: its partial-moment scratch holds
    // M / that many direction tiles)
    b->D = 8;
    for (auto *x : b->h)
        while (b->D > 1 && x->p.N % b->D) b->D >>= 1;
    for (auto *x : b->h) {
        int cand[3];
        sweep_D_candidates(x->p, cand);
        if (b->D < cand[0]) return TRT_EINVAL;   // direction counts too different to batch
    }
    // regions
    auto take = [&](size_t bytes) {
        off = (off + 255) / 256 * 256;
        char *p = base + off;
        off += bytes;
        return p;
    };
    const size_t rest = need - 4096;
    (void)rest;
    int nlev_max = 2;
    for (int s = 0; s < n; ++s) nlev_max = std::max(nlev_max, groups[s].n_levels);
    const size_t mo = max_ops(nlev_max);
    b->ctx_bytes = mo * ((size_t)n * 512 + 256);
    b->d_ctx = reinterpret_cast<unsigned char *>(take(b->ctx_bytes));
    b->meta_ints = mo * (bmeta_ints(n) + n + 64);
    b->d_meta = reinterpret_cast<int *>(take(b->meta_ints * sizeof(int)));
    b->tab_ints = mo * (2 * (size_t)n + 64);
    b->d_tab = reinterpret_cast<int *>(take(b->tab_ints * sizeof(int)));
    b->plan_cap = mo;
    b->d_plan = reinterpret_cast<PlanOp *>(take(b->plan_cap * sizeof(PlanOp)));
    b->d_dyn = reinterpret_cast<unsigned char *>(take(NCLS * (size_t)n));
    b->d_flags = reinterpret_cast<double *>(take(8 * sizeof(double) * (size_t)n));
    b->d_have_prev = reinterpret_cast<int *>(take(sizeof(int) * (size_t)n));
    if (off > opt->workspace_bytes) return TRT_ENOSPACE;
    if (cudaMallocHost(&b->h_ctx, b->ctx_bytes) != cudaSuccess ||
        cudaMallocHost(&b->h_dyn, NCLS * (size_t)n) != cudaSuccess ||
        cudaMallocHost(&b->h_flags, 8 * sizeof(double) * (size_t)n) != cudaSuccess)
        return TRT_ECUDA;
    *out = B.release();
    return TRT_OK;
}

}  // extern "C"

namespace {

// (Re)build every stage for step length dt and cycle type, lay the ops out in the regions,
// upload argument blocks, tables and planner descriptors (one copy each).
int build_all(trt_batch *b, double dt, int cycle_type)
{
    const int ids[] = {S_STEP_START, S_SWEEP, S_PHASE, S_PHASE_END, S_STEP_END,
                       S_CYCLE0 + cycle_type};
    size_t coff = 0, moff = 0, toff = 0, poff = 0;
    std::vector<int> htab;
    std::vector<PlanOp> hplan;
    // the layout (ops, offsets, grids) depends only on the slabs, the cycle type and the
    // sweep tile: graphs captured for the same key stay valid while the argument contents
    // (dt, intensity buffers) change in place
    const long key = ((long)cycle_type * 16 + b->D) * 16 + b->shape;
    if (key != b->layout_key) {
        for (auto &sg : b->stage) {
            if (sg.exec) cudaGraphExecDestroy(sg.exec);
            sg.exec = nullptr;
            sg.graph_failed = false;
        }
        b->layout_key = key;
    }
    for (auto &sg : b->stage) sg.ops.clear();
    for (int id : ids) {
        build_stage(b, id, dt, cycle_type);
        Stage &sg = b->stage[id];
        sg.plan_off = poff;
        for (auto &o : sg.ops) {
            o.ctx_off = coff;
            coff += (o.host.size() + 255) / 256 * 256;
            o.meta_off = moff;
            moff += bmeta_ints(b->n) + b->n + 64;
            o.tab_off = toff;
            toff += 2 * (size_t)b->n + 64;
            if (coff > b->ctx_bytes || moff > b->meta_ints || toff > b->tab_ints ||
                poff + 1 > b->plan_cap)
                return bfail(b, TRT_ENOSPACE, "batch plan exceeds its regions");
            std::memcpy(b->h_ctx + o.ctx_off, o.host.data(), o.host.size());
            if (htab.size() < toff) htab.resize(toff, 0);
            for (int s = 0; s < b->n; ++s) {
                htab[o.tab_off + s] = o.blocks[s];
                htab[o.tab_off + b->n + s] = o.gx[s];
            }
            PlanOp po;
            po.meta = b->d_meta + o.meta_off;
            po.blocks = b->d_tab + o.tab_off;
            po.gx = b->d_tab + o.tab_off + b->n;
            po.cls = o.cls;
            hplan.push_back(po);
            ++poff;
        }
    }
    BCK(cudaMemcpyAsync(b->d_ctx, b->h_ctx, coff, cudaMemcpyHostToDevice, b->st));
    BCK(cudaMemcpyAsync(b->d_tab, htab.data(), htab.size() * sizeof(int), cudaMemcpyHostToDevice,
                        b->st));
    BCK(cudaMemcpyAsync(b->d_plan, hplan.data(), hplan.size() * sizeof(PlanOp),
                        cudaMemcpyHostToDevice, b->st));
    BCK(cudaStreamSynchronize(b->st));   // htab / hplan are host temporaries
    b->built = true;
    b->built_dt = dt;
    return TRT_OK;
}

cudaError_t launch_op(trt_batch *b, const Op &o)
{
    const int *meta = b->d_meta + o.meta_off;
    const int N = b->n;
    const unsigned char *x = b->d_ctx + o.ctx_off;
    switch (o.kind) {
    case K_OPAC:
        return launch_opacity_b(meta, N, reinterpret_cast<const OpacityArgs *>(x), o.grid, b->st);
    case K_SWEEP:
        return launch_sweep_b(b->precision, true, b->D, b->shape, meta, N,
                              reinterpret_cast<const SweepArgs *>(x), o.grid, b->st);
    case K_FINAL:
        return launch_finalize_b(b->precision, meta, N, reinterpret_cast<const FinalizeArgs *>(x),
                                 o.grid, b->st);
    case K_LO:
        return launch_lo_solve_b(b->precision, b->max_nx, meta, N,
                                 reinterpret_cast<const LoCtx *>(x), o.grid, b->st);
    case K_RESTRICT:
        return launch_restrict_b(o.KS, meta, N, reinterpret_cast<const RestrictCtx *>(x), o.grid,
                                 b->st);
    case K_RPART:
        return launch_restrict_part_b(meta, N, reinterpret_cast<const Restrict2Ctx *>(x), o.grid,
                                      b->st);
    case K_RFINAL:
        return launch_restrict_final_b(meta, N, reinterpret_cast<const Restrict2Ctx *>(x),
                                       o.grid, b->st);
    case K_GREY:
        return launch_grey_b(b->max_nx, meta, N, reinterpret_cast<const GreyCtx *>(x), o.grid,
                             b->st);
    case K_GSUM:
        return launch_group_sum_b(meta, N, reinterpret_cast<const GroupSumArgs *>(x), o.grid,
                                  b->st);
    case K_COPY:
        return launch_copy_b(meta, N, reinterpret_cast<const CopyArgs *>(x), o.grid, b->st);
    }
    return cudaErrorInvalidValue;
}

cudaError_t enqueue_stage(trt_batch *b, Stage &sg)
{
    cudaError_t e = cudaMemcpyAsync(b->d_dyn, b->h_dyn, NCLS * (size_t)b->n, cudaMemcpyHostToDevice,
                                    b->st);
    if (e != cudaSuccess) return e;
    if (!sg.ops.empty()) {
        k_plan<<<(unsigned)sg.ops.size(), 32, 0, b->st>>>(b->d_plan + sg.plan_off,
                                                          (int)sg.ops.size(), b->d_dyn, b->n);
        e = cudaGetLastError();
        if (e != cudaSuccess) return e;
    }
    for (const auto &o : sg.ops) {
        e = launch_op(b, o);
        if (e != cudaSuccess) return e;
    }
    if (sg.d2h_flags)
        e = cudaMemcpyAsync(b->h_flags, b->d_flags, 8 * sizeof(double) * (size_t)b->n,
                            cudaMemcpyDeviceToHost, b->st);
    return e;
}

// run a stage: replay its CUDA graph once captured, else enqueue it directly (the first
// run also sets the kernels' attributes); the graph's first node reads the host's dynamic
// flags from the pinned mirror
int run_stage(trt_batch *b, int id, int &launches, bool sync)
{
    Stage &sg = b->stage[id];
    if (sg.exec)
        BCK(cudaGraphLaunch(sg.exec, b->st));
    else
        BCK(enqueue_stage(b, sg));
    launches += (int)sg.ops.size() + (sg.ops.empty() ? 0 : 1);
    if (sync) BCK(cudaStreamSynchronize(b->st));
    return TRT_OK;
}

int capture_stage(trt_batch *b, int id)
{
    Stage &sg = b->stage[id];
    if (sg.exec || sg.graph_failed) return TRT_OK;
    cudaGraph_t g = nullptr;
    if (cudaStreamBeginCapture(b->st, cudaStreamCaptureModeThreadLocal) != cudaSuccess) {
        cudaGetLastError();
        sg.graph_failed = true;
        return TRT_OK;
    }
    cudaError_t e = enqueue_stage(b, sg);
    cudaError_t e2 = cudaStreamEndCapture(b->st, &g);
    if (e != cudaSuccess || e2 != cudaSuccess || !g) {
        cudaGetLastError();
        if (g) cudaGraphDestroy(g);
        sg.graph_failed = true;
        return TRT_OK;
    }
    e = cudaGraphInstantiate(&sg.exec, g, 0);
    cudaGraphDestroy(g);
    if (e != cudaSuccess) {
        cudaGetLastError();
        sg.exec = nullptr;
        sg.graph_failed = true;
    }
    return TRT_OK;
}

}  // namespace

extern "C" {

int trt_step_batch(trt_batch *b, double dt, const trt_cycle *cyc, trt_stats *stats)
{
    if (!b) return TRT_EINVAL;
    if (!cyc || !(dt > 0) || cyc->l_max < 1 || cyc->max_outer < 1 || cyc->type < 0 ||
        cyc->type > 2)
        return bfail(b, TRT_EINVAL, "bad step arguments");
    cudaGetLastError();
    const int n = b->n;
    const bool fixed = cyc->eps < 0;
    const double eps = cyc->eps, eps_in = cyc->eps_inner;
    // argument blocks hold dt and the intensity buffers (swapped by each step that sweeps):
    // rebuild every step
    int rc = build_all(b, dt, cyc->type);
    if (rc != TRT_OK) return rc;
    for (int s = 0; s < n; ++s) BCK(ensure_lo_consts(b->h[s]->p, dt));   // LO row constants
    const int cyc_id = S_CYCLE0 + cyc->type;
    std::vector<SlabState> st(n);
    std::vector<std::vector<int>> S(n);
    for (int s = 0; s < n; ++s) {
        st[s].active = true;
        schedule(cyc->type, b->h[s]->p.nlev, S[s]);
    }
    int nk = 0;
    std::memset(b->h_dyn, 0, NCLS * (size_t)n);
    for (int s = 0; s < n; ++s) b->h_dyn[C_ALL * n + s] = 1;
    BCK(cudaMemsetAsync(b->d_flags, 0, 8 * sizeof(double) * (size_t)n, b->st));
    BCK(cudaMemsetAsync(b->d_have_prev, 0, sizeof(int) * (size_t)n, b->st));
    if ((rc = run_stage(b, S_STEP_START, nk, false)) != TRT_OK) return rc;
    bool any = true;
    while (any) {
        // outer iteration: sweep for the slabs past their s = 0 phase
        bool sweep = false;
        for (int s = 0; s < n; ++s) {
            const bool w = st[s].active && st[s].s > 0;
            b->h_dyn[C_SWEEP * n + s] = w;
            b->h_dyn[C_PHASE * n + s] = st[s].active;
            if (w) {
                sweep = true;
                st[s].n_ti++;
                st[s].swept = true;
                st[s].opac_valid = true;
            }
        }
        if (sweep && (rc = run_stage(b, S_SWEEP, nk, false)) != TRT_OK) return rc;
        if ((rc = run_stage(b, S_PHASE, nk, false)) != TRT_OK) return rc;
        for (int s = 0; s < n; ++s) {
            st[s].in_cycle = st[s].active;
            st[s].conv_out = false;
        }
        for (int l = 0; l < cyc->l_max; ++l) {
            bool anyc = false;
            for (int s = 0; s < n; ++s) {
                b->h_dyn[C_CYCLE * n + s] = st[s].in_cycle;
                b->h_dyn[C_OPAC0 * n + s] = st[s].in_cycle && !st[s].opac_valid;
                anyc = anyc || st[s].in_cycle;
            }
            if (!anyc) break;
            if (b->stage[cyc_id].exec == nullptr && b->stage[cyc_id].ops.size() && l > 0)
                capture_stage(b, cyc_id);
            if ((rc = run_stage(b, cyc_id, nk, true)) != TRT_OK) return rc;
            for (int s = 0; s < n; ++s) {
                SlabState &x = st[s];
                if (!x.in_cycle) continue;
                const Problem &p = b->h[s]->p;
                x.opac_valid = false;
                x.n_c++;
                x.n_lo += p.G + 1;
                for (int g : S[s]) x.n_lo += p.levels[g - 1] + 1;
                const double *fl = b->h_flags + 8 * (size_t)s;
                if (fl[0] != 0.0) {
                    x.status = TRT_ENUMERIC;
                    x.in_cycle = false;
                    x.active = false;
                    continue;
                }
                const bool conv_in = fl[1] <= eps_in * fl[2] && fl[3] <= eps_in * fl[4];
                x.conv_out = fl[5] <= eps * fl[2] && fl[6] <= eps * fl[4];
                if (!fixed && conv_in) x.in_cycle = false;
            }
        }
        for (int s = 0; s < n; ++s) b->h_dyn[C_PHASE_END * n + s] = st[s].active;
        if ((rc = run_stage(b, S_PHASE_END, nk, false)) != TRT_OK) return rc;
        any = false;
        for (int s = 0; s < n; ++s) {
            SlabState &x = st[s];
            if (!x.active) continue;
            ++x.s;
            if (fixed) {
                if (x.s >= cyc->max_outer) x.active = false;
            } else if (x.conv_out) {
                x.active = false;
            } else if (x.s >= cyc->max_outer) {
                x.status = TRT_ENOTCONVERGED;
                x.active = false;
            }
            any = any || x.active;
        }
        // the sweep and phase stages run once per outer iteration: capture them now
        capture_stage(b, S_PHASE);
        capture_stage(b, S_PHASE_END);
        if (sweep) capture_stage(b, S_SWEEP);
    }
    if ((rc = run_stage(b, S_STEP_END, nk, true)) != TRT_OK) return rc;
    int status = TRT_OK;
    for (int s = 0; s < n; ++s) {
        trt_handle *x = b->h[s];
        if (st[s].swept) std::swap(x->I_cur, x->I_alt);
        if (stats) {
            stats[s].n_ti = st[s].n_ti;
            stats[s].n_c = st[s].n_c;
            stats[s].n_lo = st[s].n_lo;
            stats[s].n_outer = st[s].s;
            stats[s].ms = 0;
            stats[s].status = st[s].status;
            stats[s].n_kernels = nk;
        }
        if (st[s].status != TRT_OK && status == TRT_OK) status = st[s].status;
    }
    return status;
}

trt_handle *trt_batch_slab(trt_batch *b, int s)
{
    if (!b || s < 0 || s >= b->n) return nullptr;
    return b->h[s];
}

int trt_batch_set_tile(trt_batch *b, int D, int shape)
{
    if (!b || D < 1 || D > 16 || (D & (D - 1))) return TRT_EINVAL;
    if (D == 16 && !sweep_fp32(b->precision)) return TRT_EINVAL;   // lean FP32 sweeps only
    for (auto *x : b->h) {
        int cand[3];
        sweep_D_candidates(x->p, cand);
        if (x->p.N % D || D < cand[0])
            return bfail(b, TRT_EINVAL, "D must divide every slab's N and be >= its smallest tile");
    }
    if (!sweep_tile_ok(b->precision, D, shape, true)) return TRT_EINVAL;
    b->D = D;
    b->shape = shape;
    b->built = false;
    return TRT_OK;
}

int trt_batch_sweep_time(trt_batch *b, double dt, int reps, float *ms)
{
    if (!b || !(dt > 0) || reps < 1 || !ms) return TRT_EINVAL;
    trt_cycle c{TRT_CYCLE_V, 1, 1e-8, 1e-9, 1};
    int rc = build_all(b, dt, c.type);
    if (rc != TRT_OK) return rc;
    // every slab sweeps its current intensity into its spare buffer (state unchanged but
    // the QD factors, which the sweep overwrites: restored from a copy below)
    std::memset(b->h_dyn, 0, NCLS * (size_t)b->n);
    for (int s = 0; s < b->n; ++s) b->h_dyn[C_SWEEP * b->n + s] = 1;
    Stage &sg = b->stage[S_SWEEP];
    BCK(cudaMemcpyAsync(b->d_dyn, b->h_dyn, NCLS * (size_t)b->n, cudaMemcpyHostToDevice, b->st));
    k_plan<<<(unsigned)sg.ops.size(), 32, 0, b->st>>>(b->d_plan + sg.plan_off, (int)sg.ops.size(),
                                                      b->d_dyn, b->n);
    BCK(cudaGetLastError());
    // redirect the QD-factor outputs to scratch no step reads before writing (the
    // fine-solve arrays E1 [G][nx] and F1 [G][nx+1], as trt_sweep_time does)
    for (int s = 0; s < b->n; ++s) {
        trt_handle *x = b->h[s];
        if (x->p.nx < 3) return bfail(b, TRT_EINVAL, "trt_batch_sweep_time needs n_cells >= 3");
        const size_t G = x->p.G;
        SweepArgs *a = reinterpret_cast<SweepArgs *>(b->h_ctx + sg.ops[1].ctx_off) + s;
        FinalizeArgs *f = reinterpret_cast<FinalizeArgs *>(b->h_ctx + sg.ops[2].ctx_off) + s;
        a->f = f->f = x->E1;
        a->fb0 = f->fb0 = x->F1;
        a->fbX = f->fbX = x->F1 + G;
        a->C0 = f->C0 = x->F1 + 2 * G;
        a->CX = f->CX = x->F1 + 3 * G;
    }
    BCK(cudaMemcpyAsync(b->d_ctx + sg.ops[1].ctx_off, b->h_ctx + sg.ops[1].ctx_off,
                        sg.ops[2].ctx_off + sg.ops[2].host.size() - sg.ops[1].ctx_off,
                        cudaMemcpyHostToDevice, b->st));
    BCK(launch_op(b, sg.ops[0]));   // opacities (and FP32 inputs) at the current T
    for (int r = 0; r < 1 + reps; ++r) {
        if (r == 1) {
            cudaEvent_t e0, e1;
            BCK(cudaEventCreate(&e0));
            BCK(cudaEventCreate(&e1));
            BCK(cudaEventRecord(e0, b->st));
            for (int q = 0; q < reps; ++q) {
                BCK(launch_op(b, sg.ops[1]));
                BCK(launch_op(b, sg.ops[2]));
            }
            BCK(cudaEventRecord(e1, b->st));
            BCK(cudaEventSynchronize(e1));
            float t = 0;
            BCK(cudaEventElapsedTime(&t, e0, e1));
            cudaEventDestroy(e0);
            cudaEventDestroy(e1);
            *ms = t / reps;
            break;
        }
        BCK(launch_op(b, sg.ops[1]));
        BCK(launch_op(b, sg.ops[2]));
    }
    b->built = false;
    return TRT_OK;
}

int trt_destroy_batch(trt_batch *b)
{
    delete b;
    return TRT_OK;
}

const char *trt_batch_last_error(const trt_batch *b)
{
    return b ? b->err.c_str() : "null batch";
}

}  // extern "C"
