// Host driver of the GB300 MG-GLAM field solvers: context, workspace
// pyramids, the FAS cycle (Sec. 3.2.1 of arXiv:2110.00566) replayed from
// captured CUDA graphs, and the solve entry points of include/mgglam.h.
#include <algorithm>
#include <cmath>
#include <cstdarg>
#include <cstring>

#include "ctx.cuh"

#include <functional>

namespace mg {

// ---------------------------------------------------------------------------
// errors, pointers, staging
// ---------------------------------------------------------------------------
void fail_cuda(mg_ctx *ctx, cudaError_t e, const char *call, const char *file, int line)
{
    char buf[512];
    snprintf(buf, sizeof buf, "CUDA error %d (%s) in %s at %s:%d", (int)e, cudaGetErrorString(e), call, file, line);
    if (ctx) ctx->err = buf;
}

int set_err(mg_ctx *ctx, int code, const char *fmt, ...)
{
    char buf[512];
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(buf, sizeof buf, fmt, ap);
    va_end(ap);
    if (ctx) ctx->err = buf;
    return code;
}

bool is_device_ptr(const void *p)
{
    cudaPointerAttributes a;
    if (cudaPointerGetAttributes(&a, p) != cudaSuccess) {
        cudaGetLastError();
        return false;
    }
    return a.type == cudaMemoryTypeDevice || a.type == cudaMemoryTypeManaged;
}

void *stage_in(mg_ctx *ctx, int slot, const void *p, size_t bytes, bool copy_in)
{
    if (p == nullptr) return nullptr;
    if (is_device_ptr(p)) return const_cast<void *>(p);
    if (ctx->stage_bytes[slot] < bytes) {
        if (ctx->stage[slot]) MG_CK(cudaFree(ctx->stage[slot]));
        ctx->stage[slot] = nullptr;
        ctx->stage_bytes[slot] = 0;
        MG_CK(cudaMalloc(&ctx->stage[slot], bytes));
        ctx->stage_bytes[slot] = bytes;
    }
    if (copy_in) MG_CK(cudaMemcpyAsync(ctx->stage[slot], p, bytes, cudaMemcpyHostToDevice, ctx->stream));
    return ctx->stage[slot];
}

void stage_out(mg_ctx *ctx, void *host, const void *dev, size_t bytes)
{
    if (host == dev) return;
    MG_CK(cudaMemcpyAsync(host, dev, bytes, cudaMemcpyDeviceToHost, ctx->stream));
    MG_CK(cudaStreamSynchronize(ctx->stream));
}

void enter(mg_ctx *ctx)
{
    MG_CK(cudaSetDevice(ctx->device));
    MG_CK(cudaEventRecord(ctx->ev_in, ctx->ustream));
    MG_CK(cudaStreamWaitEvent(ctx->stream, ctx->ev_in, 0));
}

void leave(mg_ctx *ctx)
{
    MG_CK(cudaEventRecord(ctx->ev_out, ctx->stream));
    MG_CK(cudaStreamWaitEvent(ctx->ustream, ctx->ev_out, 0));
}

size_t level_count(int n)
{
    size_t c = 1;
    while (n % 2 == 0 && n / 2 >= 4) {
        n /= 2;
        ++c;
    }
    return c;
}

// 2^k or 3 * 2^k cells per side, at least 8 and at most 1536: the level
// pyramid's colour arrays stay below 2^31 elements and the mesh below 2^32
// cells, the index ranges the kernels are written for (2048^3 would not fit
// one GPU's memory in any case: its FP64 finest level alone is ~340 GB)
bool valid_ng(int n)
{
    if (n < 8 || (long long)n * n * n >= (1LL << 32)) return false;
    int m = n;
    while (m % 2 == 0) m /= 2;
    return m == 1 || m == 3;
}

// ---------------------------------------------------------------------------
// workspace pyramids
// ---------------------------------------------------------------------------
static size_t al(size_t b) { return (b + 255) & ~(size_t)255; }

template <typename T>
void release_pyramid(Pyramid<T> *P)
{
    if (!P) return;
    for (auto &g : P->graphs)
        if (g.second.exec) cudaGraphExecDestroy(g.second.exec);
    if (P->block) cudaFree(P->block);
    if (P->scal) cudaFree(P->scal);
    delete P;
}

template <typename T>
static std::map<int, Pyramid<T> *> &pyr_map(mg_ctx *ctx, bool corr);
template <>
std::map<int, Pyramid<double> *> &pyr_map<double>(mg_ctx *ctx, bool corr) { return corr ? ctx->p64c : ctx->p64; }
template <>
std::map<int, Pyramid<float> *> &pyr_map<float>(mg_ctx *ctx, bool corr) { return corr ? ctx->p32c : ctx->p32; }

template <typename T>
Pyramid<T> *alloc_pyramid(mg_ctx *ctx, int n, bool correction)
{
    auto *P = new Pyramid<T>();
    P->n0 = n;
    P->nlev = (int)level_count(n);
    P->correction = correction;
    P->L.resize(P->nlev);
    size_t total = 0;
    const int per_level = 10 + (correction ? 2 : 0);
    for (int l = 0; l < P->nlev; ++l) {
        const long long nl = n >> l;
        total += per_level * al(sizeof(T) * (size_t)(nl * nl * nl / 2));
    }
    // reduction partials: the (m, j) block plane of the finest level may
    // exceed MAX_RED_BLOCKS on very large meshes
    const long long plane = (long long)((n / 2 + 31) / 32) * ((n + 7) / 8);
    const int cap = (int)std::max<long long>(MAX_RED_BLOCKS, plane);
    const size_t small = al(sizeof(LevScal) * P->nlev) + al(sizeof(OpK<T>)) + al(sizeof(OpK<double>)) +
                         al(sizeof(double) * 4 * (size_t)cap) + al(sizeof(unsigned int));
    cudaError_t e = cudaMalloc(&P->block, total);
    if (e != cudaSuccess) {
        delete P;
        fail_cuda(ctx, e, "cudaMalloc(pyramid)", __FILE__, __LINE__);
        throw CudaFail{MG_ERR_OOM};
    }
    e = cudaMalloc((void **)&P->scal, small);
    if (e != cudaSuccess) {
        cudaFree(P->block);
        delete P;
        fail_cuda(ctx, e, "cudaMalloc(scalars)", __FILE__, __LINE__);
        throw CudaFail{MG_ERR_OOM};
    }
    MG_CK(cudaMemsetAsync(P->scal, 0, small, ctx->stream));
    char *sp = (char *)P->scal + al(sizeof(LevScal) * P->nlev);
    P->opT = (OpK<T> *)sp;
    sp += al(sizeof(OpK<T>));
    P->opD = (OpK<double> *)sp;
    sp += al(sizeof(OpK<double>));
    P->rb.partials = (double *)sp;
    sp += al(sizeof(double) * 4 * (size_t)cap);
    P->rb.counter = (unsigned int *)sp;
    P->rb.cap = cap;
    char *bp = (char *)P->block;
    for (int l = 0; l < P->nlev; ++l) {
        LevArrays<T> &L = P->L[l];
        L.n = n >> l;
        L.half = L.n / 2;
        L.ncol = (long long)L.n * L.n * L.n / 2;
        L.h = (double)(1 << l);
        const size_t b = al(sizeof(T) * (size_t)L.ncol);
        auto take = [&]() {
            T *p = (T *)bp;
            bp += b;
            return p;
        };
        for (int q = 0; q < 2; ++q)
            for (int c = 0; c < 2; ++c) L.u[q][c] = take();
        L.cur[0] = L.cur[1] = 0;
        for (int c = 0; c < 2; ++c) L.s[c] = take();
        for (int c = 0; c < 2; ++c) L.fbuf[c] = take();
        for (int c = 0; c < 2; ++c) L.ur[c] = take();
        for (int c = 0; c < 2; ++c) L.base[c] = correction ? take() : nullptr;
        for (int c = 0; c < 2; ++c) L.f[c] = (l == 0 && !correction) ? nullptr : L.fbuf[c];
        L.sc = P->scal + l;
    }
    P->bytes = total + small;
    P->block_bytes = total;
    return P;
}

template <typename T>
Pyramid<T> *get_pyramid(mg_ctx *ctx, int n, bool correction)
{
    auto &mp = pyr_map<T>(ctx, correction);
    auto it = mp.find(n);
    if (it != mp.end()) return it->second;
    Pyramid<T> *P = alloc_pyramid<T>(ctx, n, correction);
    mp[n] = P;
    return P;
}

template Pyramid<double> *get_pyramid<double>(mg_ctx *, int, bool);
template Pyramid<float> *get_pyramid<float>(mg_ctx *, int, bool);
template Pyramid<double> *alloc_pyramid<double>(mg_ctx *, int, bool);
template Pyramid<float> *alloc_pyramid<float>(mg_ctx *, int, bool);
template void release_pyramid<double>(Pyramid<double> *);
template void release_pyramid<float>(Pyramid<float> *);

// ---------------------------------------------------------------------------
// the FAS cycle (Sec. 3.2.1): pre-smooth, fused residual + restriction,
// coarse source, recursion (V: once, W: twice, F: F then V), prolongation
// with correction, post-smooth; the coarsest level is solved in one CTA.
// ---------------------------------------------------------------------------
// one half-sweep; on the finest level with profiling on, bracketed by a
// pair of events (recorded as graph nodes when the stream is capturing)
template <typename T>
static void smooth_half(mg_ctx *ctx, Pyramid<T> &P, int l, int colour)
{
    cudaStream_t st = ctx->stream;
    LevArrays<T> &L = P.L[l];
    const bool prof = ctx->prof_on && l == 0;
    // inside a capture the events must become external event-record nodes
    // (timestamps); outside a capture the external flag is not allowed
    unsigned int flags = cudaEventRecordDefault;
    if (prof) {
        cudaStreamCaptureStatus cs = cudaStreamCaptureStatusNone;
        MG_CK(cudaStreamIsCapturing(st, &cs));
        if (cs == cudaStreamCaptureStatusActive) flags = cudaEventRecordExternal;
    }
    if (prof) {
        const size_t need = 2 * (size_t)(ctx->prof_k + 1);
        while (ctx->pev.size() < need) {
            cudaEvent_t e;
            MG_CK(cudaEventCreate(&e));
            ctx->pev.push_back(e);
        }
        MG_CK(cudaEventRecordWithFlags(ctx->pev[2 * ctx->prof_k], st, flags));
    }
    launch_smooth<T>(L, &L, P.opT, colour, st);
    if (prof) {
        MG_CK(cudaEventRecordWithFlags(ctx->pev[2 * ctx->prof_k + 1], st, flags));
        ++ctx->prof_k;
    }
}

template <typename T>
static void run_cycle(mg_ctx *ctx, Pyramid<T> &P, const mg_opts &o, int l, int type)
{
    cudaStream_t st = ctx->stream;
    LevArrays<T> &L = P.L[l];
    if (l == P.nlev - 1) {
        launch_coarsest<T>(L, P.opD, o.coarse_sweeps, st);
        return;
    }
    for (int q = 0; q < o.pre; ++q) {
        smooth_half(ctx, P, l, 0);
        smooth_half(ctx, P, l, 1);
    }
    launch_resid_restrict<T>(L, P.L[l + 1], P.opT, P.rb, st);
    launch_coarse_source<T>(L, P.L[l + 1], P.opT, P.rb, st);
    const int visits = type == MG_CYCLE_W ? 2 : 1;
    for (int v = 0; v < visits; ++v) run_cycle(ctx, P, o, l + 1, type);
    if (type == MG_CYCLE_F) run_cycle(ctx, P, o, l + 1, MG_CYCLE_V);
    launch_prolong<T>(L, P.L[l + 1], st);
    for (int q = 0; q < o.post; ++q) {
        smooth_half(ctx, P, l, 0);
        smooth_half(ctx, P, l, 1);
    }
}

// kernels launched by one cycle (run_cycle) plus the residual norm
template <typename T>
static long long cycle_launches(const Pyramid<T> &P, const mg_opts &o, int l, int type)
{
    if (l == P.nlev - 1) return 1;
    long long c = 2LL * (o.pre + o.post) + 2 + prolong_kernels<T>(P.L[l]);
    const int visits = type == MG_CYCLE_W ? 2 : 1;
    for (int v = 0; v < visits; ++v) c += cycle_launches(P, o, l + 1, type);
    if (type == MG_CYCLE_F) c += cycle_launches(P, o, l + 1, MG_CYCLE_V);
    return c;
}

// device time of the finest-level smoother launches of the last cycle
static double prof_collect(mg_ctx *ctx)
{
    double ms = 0.0;
    for (int k = 0; k < ctx->prof_k; ++k) {
        float t = 0.f;
        MG_CK(cudaEventElapsedTime(&t, ctx->pev[2 * k], ctx->pev[2 * k + 1]));
        ms += t;
    }
    return ms;
}

template <typename T>
static long long cycle_updates(const Pyramid<T> &P, const mg_opts &o, int l, int type)
{
    const long long cells = 2LL * P.L[l].ncol;
    if (l == P.nlev - 1) return (long long)o.coarse_sweeps * cells;
    long long u = (long long)(o.pre + o.post) * cells;
    const int visits = type == MG_CYCLE_W ? 2 : 1;
    for (int v = 0; v < visits; ++v) u += cycle_updates(P, o, l + 1, type);
    if (type == MG_CYCLE_F) u += cycle_updates(P, o, l + 1, MG_CYCLE_V);
    return u;
}

// One cycle followed by the finest residual norm, from a captured graph
// when use_graph is set (one graph per pointer state of the ping-pong
// buffers; the state returns to itself when pre + post is even).
// (norm = false: the cycle alone, for the inner cycles of the mixed solve,
// whose convergence is judged by the FP64 defect)
template <typename T>
static void cycle_and_norm(mg_ctx *ctx, Pyramid<T> &P, const mg_opts &o, bool norm = true)
{
    auto record = [&]() {
        ctx->prof_k = 0;
        run_cycle(ctx, P, o, 0, o.cycle);
        if (norm) launch_resid_norm<T>(P.L[0], P.opT, P.rb, ctx->stream);
    };
    if (!o.use_graph) {
        record();
        return;
    }
    CycleKey key{P.state(), o.pre, o.post, o.cycle, o.coarse_sweeps, P.nlev, ctx->prof_on, norm ? 1 : 0, P.L[0].model};
    auto it = P.graphs.find(key);
    if (it == P.graphs.end()) {
        const std::vector<int> pre_state = P.state();
        cudaGraph_t g = nullptr;
        MG_CK(cudaStreamBeginCapture(ctx->stream, cudaStreamCaptureModeThreadLocal));
        record();
        MG_CK(cudaStreamEndCapture(ctx->stream, &g));
        GraphEntry e;
        e.post_state = P.state();
        e.nprof = ctx->prof_k;
        MG_CK(cudaGraphInstantiate(&e.exec, g, 0));
        MG_CK(cudaGraphDestroy(g));
        P.set_state(pre_state);
        it = P.graphs.emplace(key, e).first;
    }
    MG_CK(cudaGraphLaunch(it->second.exec, ctx->stream));
    P.set_state(it->second.post_state);
    ctx->prof_k = it->second.nprof;
}

static void read_scal(mg_ctx *ctx, const LevScal *d, LevScal *h)
{
    MG_CK(cudaMemcpyAsync(ctx->hpin, d, sizeof(LevScal), cudaMemcpyDeviceToHost, ctx->stream));
    MG_CK(cudaStreamSynchronize(ctx->stream));
    memcpy(h, ctx->hpin, sizeof(LevScal));
}

template <typename T>
static void upload_op(mg_ctx *ctx, Pyramid<T> &P, const ModelDesc &md)
{
    static thread_local OpK<T> hT;
    static thread_local OpK<double> hD;
    hT = make_opk<T>(md.model, md.alpha, md.nkmo, md.gamma, md.bterm);
    hD = make_opk<double>(md.model, md.alpha, md.nkmo, md.gamma, md.bterm);
    MG_CK(cudaMemcpyAsync(P.opT, &hT, sizeof hT, cudaMemcpyHostToDevice, ctx->stream));
    MG_CK(cudaMemcpyAsync(P.opD, &hD, sizeof hD, cudaMemcpyHostToDevice, ctx->stream));
    MG_CK(cudaStreamSynchronize(ctx->stream));
    for (auto &L : P.L) L.model = md.model;
}

// Plain solve: every level in the storage precision T (FP64 for the
// library's MG_PREC_FP64).  delta, phi: device pointers.
template <typename T>
static int solve_plain(mg_ctx *ctx, int n, const ModelDesc &md, const double *delta, double *phi, const mg_opts &o,
                       mg_stats *st)
{
    Pyramid<T> &P = *get_pyramid<T>(ctx, n, false);
    cudaStream_t s = ctx->stream;
    const long long cnt = (long long)n * n * n;
    upload_op(ctx, P, md);
    MG_CK(cudaMemsetAsync(P.scal, 0, sizeof(LevScal) * P.nlev, s));
    MG_CK(cudaEventRecord(ctx->t0, s));
    LevScal *s0 = P.scal;
    // source prep: <delta>, s = coef (delta - <delta>), eps_ref, density pyramid
    launch_mean_nat(delta, cnt, &s0->mean, P.rb, s);
    launch_split<T>(delta, n, P.L[0].s, md.s_coef, &s0->mean, s);
    launch_rms_nat(delta, cnt, md.eref_coef, &s0->mean, &s0->aux, P.rb, s);
    for (int l = 0; l + 1 < P.nlev; ++l) launch_restrict_plain<T>(P.L[l].s, P.L[l].n, P.L[l + 1].s, s);
    LevArrays<T> &L0 = P.L[0];
    if (o.warm_start) {
        T *dst[2] = {L0.U(0), L0.U(1)};
        launch_split<T>(phi, n, dst, 1.0, nullptr, s);
    } else {
        MG_CK(cudaMemsetAsync(L0.U(0), 0, sizeof(T) * L0.ncol, s));
        MG_CK(cudaMemsetAsync(L0.U(1), 0, sizeof(T) * L0.ncol, s));
    }
    launch_resid_norm<T>(L0, P.opT, P.rb, s, nullptr, !o.warm_start);
    LevScal h;
    read_scal(ctx, s0, &h);
    const double eps_ref = h.aux;
    double eps = std::sqrt(std::fmax(h.eps2, 0.0));
    mg_stats loc{};
    loc.eps_ref = eps_ref;
    loc.eps[0] = eps;
    loc.n_eps = 1;
    if (!std::isfinite(eps) || !std::isfinite(eps_ref)) {
        if (st) *st = loc;
        return set_err(ctx, MG_ERR_NONFINITE, "non-finite initial residual (delta has NaN/Inf?)");
    }
    const long long per_cycle = cycle_updates(P, o, 0, o.cycle);
    int cyc = 0, norms = 0;
    bool conv = eps <= o.rtol * eps_ref + o.atol;
    // The finest residual norm costs about two half-sweeps: it is measured
    // after the first cycle, then whenever the residual predicted with half
    // the observed per-cycle reduction rate reaches the tolerance, and at
    // least every third cycle.  The optimistic prediction never skips a cycle
    // at which the real residual has reached the tolerance (as long as the
    // rate does not improve more than twofold), so no cycle is wasted;
    // unmeasured cycles take c from their own residual/restriction pass.
    // Convergence is only declared on a measured residual.
    const double target = o.rtol * eps_ref + o.atol;
    double rho = 0.05, eps_meas = eps;
    int since = 0;
    while (!conv && cyc < o.max_cycles) {
        ++since;
        const double predicted = eps_meas * std::pow(rho, since);
        const bool measure = cyc == 0 || predicted <= target || since >= 3 || cyc + 1 == o.max_cycles;
        cycle_and_norm(ctx, P, o, measure);
        ++cyc;
        if (ctx->prof_on) {
            MG_CK(cudaStreamSynchronize(s));
            loc.fine_smooth_ms += prof_collect(ctx);
            loc.fine_smooth_launches += ctx->prof_k;
        }
        if (!measure) continue;
        ++norms;
        read_scal(ctx, s0, &h);
        eps = std::sqrt(std::fmax(h.eps2, 0.0));
        if (eps > 0 && eps < eps_meas)
            rho = std::min(0.9, std::max(1e-4, 0.5 * std::pow(eps / eps_meas, 1.0 / since)));
        else
            rho = 0.9;
        eps_meas = eps;
        since = 0;
        if (loc.n_eps < 65) loc.eps[loc.n_eps++] = eps;
        if (!std::isfinite(eps)) {
            loc.cycles = cyc;
            if (st) *st = loc;
            return set_err(ctx, MG_ERR_NONFINITE, "non-finite residual after cycle %d", cyc);
        }
        conv = eps <= o.rtol * eps_ref + o.atol;
    }
    const double c_final = h.c, clamps = h.clamps;
    // gauge <phi> = 0, back to the natural layout
    T *src[2] = {L0.U(0), L0.U(1)};
    launch_mean_split<T>(src, L0.ncol, &s0->mean, P.rb, s);
    launch_merge<T>(src, n, phi, &s0->mean, s);
    MG_CK(cudaEventRecord(ctx->t1, s));
    read_scal(ctx, s0, &h);
    float ms = 0.f;
    MG_CK(cudaEventElapsedTime(&ms, ctx->t0, ctx->t1));
    loc.cycles = cyc;
    loc.c_final = c_final;
    loc.mean_shift = h.mean;
    loc.sqrt_clamps = (long long)clamps;
    loc.ms = ms;
    loc.cell_updates = per_cycle * cyc;
    loc.kernel_launches = (P.nlev - 1) + 6 + (o.warm_start ? 1 : 0) + cyc * cycle_launches(P, o, 0, o.cycle) + norms;
    const int rc = conv ? MG_OK : MG_WARN_NOT_CONVERGED;
    loc.status = rc;
    if (st) *st = loc;
    if (!conv) set_err(ctx, rc, "not converged after %d cycles: eps/eps_ref = %g", cyc, eps / eps_ref);
    return rc;
}

// Block shape of the FP32 four-cell smoother per level (threads along a row:
// 8, 16, 32 or 64; 256 per block), picked once per pyramid by timing
// half-sweeps on the level's own arrays (into the alternate buffer) before
// any cycle is captured.  Levels below 64^3 keep the default.
static float time_launch(mg_ctx *ctx, const std::function<bool(int)> &launch)
{
    cudaStream_t s = ctx->stream;
    float t = 1e30f;
    for (int r = 0; r < 3; ++r) {
        MG_CK(cudaEventRecord(ctx->t0, s));
        if (!launch(r & 1)) return 1e30f;
        MG_CK(cudaEventRecord(ctx->t1, s));
        MG_CK(cudaEventSynchronize(ctx->t1));
        float ms = 0.f;
        MG_CK(cudaEventElapsedTime(&ms, ctx->t0, ctx->t1));
        t = std::min(t, ms);
    }
    MG_CK(cudaGetLastError());
    return t;
}

// per FP32 level: the gathering kernel's block shape, and whether a
// streaming variant beats it (each candidate timed on both colours into the
// alternate buffers, so the level's state is untouched)
static void tune_smooth4(mg_ctx *ctx, Pyramid<float> &P)
{
    cudaStream_t s = ctx->stream;
    for (auto &L : P.L) {
        if (L.qbx != 0 || L.n < 64) continue;
        int best = 0, best_z = 1;
        float best_ms = 1e30f;
        auto pin = ctx->fp32_shape.find(L.n);
        const bool pinned = pin != ctx->fp32_shape.end() && launch_smooth4_shape(L, P.opT, 0, pin->second.first, 1, s);
        if (pinned) {
            // pinned shape: still timed, so that a streaming variant must beat it
            best = pin->second.first;
            best_z = pin->second.second;
            best_ms = time_launch(ctx, [&](int c) { return launch_smooth4_shape(L, P.opT, c, best, best_z, s); });
        }
        for (int bx : {8, 16, 32, 64}) {
            if (pinned) break;
            if (bx > L.half / 4) continue;
            if (!launch_smooth4_shape(L, P.opT, 0, bx, 1, s)) break;
            for (int zc : {1, 2, 4, 8}) {
                if (zc > 1 && L.n < 128) break;
                const float t =
                    time_launch(ctx, [&](int c) { return launch_smooth4_shape(L, P.opT, c, bx, zc, s); });
                if (t < best_ms) {
                    best_ms = t;
                    best = bx;
                    best_z = zc;
                }
            }
        }
        L.qbx = best > 0 ? best : -1;
        L.qz = best_z;
        L.qstream = -1;
        if (!stream_eligible(L) || ctx->fp32_smoother < 0) continue;
        if (ctx->fp32_smoother > 0) {
            stream_setup();
            L.qstream = ctx->fp32_smoother;
            continue;
        }
        const LevK<float> K = make_levk<float>(L.n, L.h);
        for (int v = 1; v <= stream_variants(); ++v) {
            const float t = time_launch(ctx, [&](int c) {
                return launch_smooth_stream(L, K, P.opT, c, 1 - L.cur[c], v, s);
            });
            if (t < best_ms) {
                best_ms = t;
                L.qstream = v;
            }
        }
    }
}

// Mixed precision (defect correction / iterative refinement): the FP64
// master field u and the FP64 finest-level defect d = L(u) drive FP32 FAS
// cycles on the correction e, which solve L(u + e) - L(u) = -d with the base
// field b = fl32(u) frozen (operator N(b + e) - N(b) in cancellation-free
// form, so the FP32 corrections keep their own relative precision); then
// u += e and the defect is recomputed in FP64.  Norms, the compatibility
// constants and the coarsest solve are FP64.
int solve_mixed(mg_ctx *ctx, int n, const ModelDesc &md, const double *delta, double *phi, const mg_opts &o,
                mg_stats *st)
{
    Pyramid<double> &P64 = *get_pyramid<double>(ctx, n, false);
    Pyramid<float> &P32 = *get_pyramid<float>(ctx, n, true);
    cudaStream_t s = ctx->stream;
    const long long cnt = (long long)n * n * n;
    upload_op(ctx, P64, md);
    upload_op(ctx, P32, md);
    tune_smooth4(ctx, P32);
    MG_CK(cudaMemsetAsync(P64.scal, 0, sizeof(LevScal) * P64.nlev, s));
    MG_CK(cudaMemsetAsync(P32.scal, 0, sizeof(LevScal) * P32.nlev, s));
    MG_CK(cudaEventRecord(ctx->t0, s));
    LevScal *s0 = P64.scal;
    LevArrays<double> &U64 = P64.L[0];
    LevArrays<float> &E0 = P32.L[0];
    // source prep in FP64, density pyramid in FP32
    launch_mean_nat(delta, cnt, &s0->mean, P64.rb, s);
    launch_split<double>(delta, n, U64.s, md.s_coef, &s0->mean, s);
    launch_rms_nat(delta, cnt, md.eref_coef, &s0->mean, &s0->aux, P64.rb, s);
    launch_convert<float, double>(E0.s, U64.s, U64.ncol, s);
    for (int l = 0; l + 1 < P32.nlev; ++l) launch_restrict_plain<float>(P32.L[l].s, P32.L[l].n, P32.L[l + 1].s, s);
    double *Uu[2] = {U64.U(0), U64.U(1)};
    if (o.warm_start) {
        launch_split<double>(phi, n, Uu, 1.0, nullptr, s);
    } else {
        MG_CK(cudaMemsetAsync(Uu[0], 0, sizeof(double) * U64.ncol, s));
        MG_CK(cudaMemsetAsync(Uu[1], 0, sizeof(double) * U64.ncol, s));
    }
    float *D[2] = {E0.fbuf[0], E0.fbuf[1]};
    launch_resid_norm<double>(U64, P64.opT, P64.rb, s, D, !o.warm_start);
    LevScal h;
    read_scal(ctx, s0, &h);
    const double eps_ref = h.aux;
    double eps = std::sqrt(std::fmax(h.eps2, 0.0));
    mg_stats loc{};
    loc.eps_ref = eps_ref;
    loc.eps[0] = eps;
    loc.n_eps = 1;
    if (!std::isfinite(eps) || !std::isfinite(eps_ref)) {
        if (st) *st = loc;
        return set_err(ctx, MG_ERR_NONFINITE, "non-finite initial residual (delta has NaN/Inf?)");
    }
    // inner FP32 cycles per FP64 defect: fixed, or (inner_cycles = 0) as
    // many as the observed per-cycle reduction rho needs to reach the
    // tolerance, 1..MAX_ADAPT_INNER (rho = 0.1 assumed before the first
    // measurement); the FP32 correction resolves about 1e-6 of itself, so
    // longer inner runs gain nothing
    constexpr int MAX_ADAPT_INNER = 4;
    double rho = 0.1;
    const long long per_cycle = cycle_updates(P32, o, 0, o.cycle);
    const long long per_launch = cycle_launches(P32, o, 0, o.cycle) + 1;
    long long launches = 6 + (P32.nlev - 1) + (o.warm_start ? 1 : 0);
    int cyc = 0, outer = 0;
    bool conv = eps <= o.rtol * eps_ref + o.atol;
    while (!conv && cyc < o.max_cycles) {
        // base field b = fl32(u) on every level, correction e = 0
        launch_convert<float, double>(E0.base, Uu, U64.ncol, s);
        for (int l = 0; l + 1 < P32.nlev; ++l)
            launch_restrict_plain<float>(P32.L[l].base, P32.L[l].n, P32.L[l + 1].base, s);
        launch_set_corr_scalars(P32.scal, s0, P32.nlev, s);
        MG_CK(cudaMemsetAsync(E0.U(0), 0, sizeof(float) * E0.ncol, s));
        MG_CK(cudaMemsetAsync(E0.U(1), 0, sizeof(float) * E0.ncol, s));
        int inner = o.inner_cycles;
        if (inner <= 0) {
            const double target = o.rtol * eps_ref + o.atol;
            // 25% margin: one more FP32 cycle is cheaper than one more FP64 defect
            const double need = (eps > target && target > 0) ? std::log(target / eps) / std::log(rho) : 1.0;
            inner = (int)std::min<double>(MAX_ADAPT_INNER, std::max(1.0, std::ceil(1.25 * need - 1e-9)));
        }
        const double eps_before = eps;
        int ran = 0;
        for (int k = 0; k < inner && cyc < o.max_cycles; ++k, ++ran) {
            cycle_and_norm(ctx, P32, o, false);
            ++cyc;
            launches += per_launch - 1;
            if (ctx->prof_on) {
                MG_CK(cudaStreamSynchronize(s));
                loc.fine_smooth_ms += prof_collect(ctx);
                loc.fine_smooth_launches += ctx->prof_k;
            }
        }
        float *Ee[2] = {E0.U(0), E0.U(1)};
        launch_add_correction(Uu, Ee, U64.ncol, s);
        launch_resid_norm<double>(U64, P64.opT, P64.rb, s, D);
        launches += 3 + (P32.nlev - 1) + 1;
        ++outer;
        read_scal(ctx, s0, &h);
        eps = std::sqrt(std::fmax(h.eps2, 0.0));
        if (loc.n_eps < 65) loc.eps[loc.n_eps++] = eps;
        if (!std::isfinite(eps)) {
            loc.cycles = cyc;
            if (st) *st = loc;
            return set_err(ctx, MG_ERR_NONFINITE, "non-finite residual after correction %d", outer);
        }
        conv = eps <= o.rtol * eps_ref + o.atol;
        if (ran > 0 && eps > 0 && eps < eps_before)
            rho = std::min(0.9, std::max(1e-3, std::pow(eps / eps_before, 1.0 / ran)));
    }
    for (const auto &L : P32.L)
        if (L.qstream > 0) {
            const int f = stream_timeout_flag(s, true);
            if (f != 0) {
                loc.cycles = cyc;
                if (st) *st = loc;
                return f < 0 ? set_err(ctx, MG_ERR_CUDA, "reading the streaming smoother's flag failed")
                             : set_err(ctx, MG_ERR_TIMEOUT, "a bounded wait of the streaming smoother gave up");
            }
            break;
        }
    const double c_final = h.c, clamps = h.clamps;
    launch_mean_split<double>(Uu, U64.ncol, &s0->mean, P64.rb, s);
    launch_merge<double>(Uu, n, phi, &s0->mean, s);
    MG_CK(cudaEventRecord(ctx->t1, s));
    read_scal(ctx, s0, &h);
    float ms = 0.f;
    MG_CK(cudaEventElapsedTime(&ms, ctx->t0, ctx->t1));
    loc.cycles = cyc;
    loc.c_final = c_final;
    loc.mean_shift = h.mean;
    loc.sqrt_clamps = (long long)clamps;
    loc.ms = ms;
    loc.cell_updates = per_cycle * cyc;
    loc.kernel_launches = launches;
    const int rc = conv ? MG_OK : MG_WARN_NOT_CONVERGED;
    loc.status = rc;
    if (st) *st = loc;
    if (!conv) set_err(ctx, rc, "not converged after %d FP32 cycles: eps/eps_ref = %g", cyc, eps / eps_ref);
    return rc;
}

int check_opts(mg_ctx *ctx, const mg_opts &o)
{
    if (o.pre < 0 || o.post < 0 || o.pre + o.post == 0 || o.max_cycles < 0 || o.max_cycles > 64)
        return set_err(ctx, MG_ERR_ARG, "bad pre/post/max_cycles");
    if (o.cycle < 0 || o.cycle > 2) return set_err(ctx, MG_ERR_ARG, "bad cycle type %d", o.cycle);
    if (o.precision < 0 || o.precision > 1) return set_err(ctx, MG_ERR_ARG, "bad precision %d", o.precision);
    if (o.coarse_sweeps < 1) return set_err(ctx, MG_ERR_ARG, "coarse_sweeps must be >= 1");
    if (!(o.rtol >= 0) || !(o.atol >= 0)) return set_err(ctx, MG_ERR_ARG, "bad rtol/atol");
    return MG_OK;
}

static double beta_dgp(double a, double om, double rc)
{
    const double orc = 1.0 / (4.0 * rc * rc);
    const double oma = om / (a * a * a), ol = 1.0 - om;
    return 1.0 + (oma + 2.0 * ol) / (2.0 * std::sqrt(orc * (oma + ol)));
}

// run a model solve on device arrays, staging host arrays
static int solve_any(mg_ctx *ctx, int n, const ModelDesc &md, const double *delta_in, double *phi_io,
                     const mg_opts &o, mg_stats *st)
{
    const size_t bytes = sizeof(double) * (size_t)n * n * n;
    const double *delta = (const double *)stage_in(ctx, 0, delta_in, bytes, true);
    double *phi = (double *)stage_in(ctx, 1, phi_io, bytes, o.warm_start != 0);
    int rc;
    if (o.precision == MG_PREC_FP64)
        rc = solve_plain<double>(ctx, n, md, delta, phi, o, st);
    else
        rc = solve_mixed(ctx, n, md, delta, phi, o, st);
    if (rc >= 0) stage_out(ctx, phi_io, phi, bytes);
    return rc;
}

// Kmouflage operator description (the model's constants in code units)
static ModelDesc kmo_desc(const mg_grid &g, const mg_kmo_params &p)
{
    const double a = g.a;
    double gam = p.n * p.k0;
    for (int q = 0; q < p.n - 1; ++q) gam *= 1.0 / (2.0 * a * a * p.lambda * p.lambda);
    const double ct = 2997.92458 * g.ng / g.box_mpch;   // c~ = (c/H0) N / L
    const double coef = 3.0 * p.beta_kmo * p.A_bar * g.omega_m / a / ct;
    const double b = p.phibar_prime_over_h0 * p.phibar_prime_over_h0;
    return ModelDesc{1, 0.0, p.n, gam, b, coef, coef};
}

// Kmouflage solve on device arrays (used by the particle-mesh step)
int solve_kmo_dev(mg_ctx *ctx, const mg_grid &g, const mg_kmo_params &p, const double *delta, double *phi,
                  const mg_opts &o, mg_stats *st)
{
    const ModelDesc md = kmo_desc(g, p);
    if (o.precision == MG_PREC_FP64) return solve_plain<double>(ctx, g.ng, md, delta, phi, o, st);
    return solve_mixed(ctx, g.ng, md, delta, phi, o, st);
}

// nDGP solve on device arrays (used by the particle-mesh step)
int solve_dgp_dev(mg_ctx *ctx, int n, double a, double om, double rc, const double *delta, double *phi,
                  const mg_opts &o, mg_stats *st)
{
    const double beta = beta_dgp(a, om, rc);
    const double alpha = 3.0 * beta * a * a / (rc * rc);
    ModelDesc md{0, alpha, 0, 0.0, 0.0, (alpha / beta) * om / a, om / (a * beta)};
    if (o.precision == MG_PREC_FP64) return solve_plain<double>(ctx, n, md, delta, phi, o, st);
    return solve_mixed(ctx, n, md, delta, phi, o, st);
}

}  // namespace mg

using namespace mg;

// ===========================================================================
// C-ABI
// ===========================================================================
extern "C" {

void mg_opts_default(mg_opts *o)
{
    if (!o) return;
    memset(o, 0, sizeof *o);
    o->pre = 2;
    o->post = 2;
    o->max_cycles = 30;
    o->cycle = MG_CYCLE_V;
    o->precision = MG_PREC_FP64;
    o->rtol = 1e-8;
    o->atol = 0.0;
    o->warm_start = 0;
    o->coarse_sweeps = 16;
    o->use_graph = 1;
    o->inner_cycles = 0;
}

int mg_ctx_create(mg_ctx **out, int device, void *cuda_stream)
{
    if (!out) return MG_ERR_ARG;
    *out = nullptr;
    mg_ctx *ctx = new mg_ctx();
    ctx->device = device;
    try {
        MG_CK(cudaSetDevice(device));
        MG_CK(cudaStreamCreateWithFlags(&ctx->stream, cudaStreamNonBlocking));
        ctx->ustream = (cudaStream_t)cuda_stream;
        MG_CK(cudaEventCreateWithFlags(&ctx->ev_in, cudaEventDisableTiming));
        MG_CK(cudaEventCreateWithFlags(&ctx->ev_out, cudaEventDisableTiming));
        MG_CK(cudaEventCreate(&ctx->t0));
        MG_CK(cudaEventCreate(&ctx->t1));
        MG_CK(cudaMallocHost((void **)&ctx->hpin, 64 * sizeof(double)));
        MG_CK(cudaMalloc((void **)&ctx->dscratch, 64 * sizeof(double) + sizeof(double) * 4 * MAX_RED_BLOCKS +
                                                      256));
        MG_CK(cudaMemset(ctx->dscratch, 0, 64 * sizeof(double) + sizeof(double) * 4 * MAX_RED_BLOCKS + 256));
        ctx->rb.partials = ctx->dscratch + 64;
        ctx->rb.counter = (unsigned int *)(ctx->rb.partials + 4 * MAX_RED_BLOCKS);
        ctx->rb.cap = MAX_RED_BLOCKS;
    } catch (CudaFail &f) {
        int code = f.code;
        mg_ctx_destroy(ctx);
        return code;
    }
    *out = ctx;
    return MG_OK;
}

void mg_pm_free(mg_ctx *ctx);

void mg_ctx_destroy(mg_ctx *ctx)
{
    if (!ctx) return;
    cudaSetDevice(ctx->device);
    if (ctx->stream) cudaStreamSynchronize(ctx->stream);
    for (auto &p : ctx->p64) release_pyramid(p.second);
    for (auto &p : ctx->p32) release_pyramid(p.second);
    for (auto &p : ctx->p64c) release_pyramid(p.second);
    for (auto &p : ctx->p32c) release_pyramid(p.second);
    batch_free(ctx);
    adj_release(ctx);
    dpm_release(ctx);
    mg_pm_free(ctx);
    for (int q = 0; q < mg_ctx::NSTAGE; ++q)
        if (ctx->stage[q]) cudaFree(ctx->stage[q]);
    for (auto e : ctx->pev) cudaEventDestroy(e);
    if (ctx->hpin) cudaFreeHost(ctx->hpin);
    if (ctx->dscratch) cudaFree(ctx->dscratch);
    if (ctx->ev_in) cudaEventDestroy(ctx->ev_in);
    if (ctx->ev_out) cudaEventDestroy(ctx->ev_out);
    if (ctx->t0) cudaEventDestroy(ctx->t0);
    if (ctx->t1) cudaEventDestroy(ctx->t1);
    if (ctx->stream) cudaStreamDestroy(ctx->stream);
    delete ctx;
}

const char *mg_last_error_string(const mg_ctx *ctx)
{
    if (!ctx) return "null context";
    return ctx->err.c_str();
}

int mg_ctx_set_profiling(mg_ctx *ctx, int on)
{
    if (!ctx) return MG_ERR_ARG;
    ctx->prof_on = on ? 1 : 0;
    return MG_OK;
}

int mg_fp32_smoother_variants(void) { return stream_variants(); }

// forget the FP32 smoother tuning and the graphs that captured it
static void reset_fp32_tuning(mg_ctx *ctx)
{
    for (auto *m : {&ctx->p32, &ctx->p32c})
        for (auto &kv : *m) {
            for (auto &l : kv.second->L) {
                l.qbx = l.qstream = 0;
                l.qz = 1;
            }
            for (auto &g : kv.second->graphs)
                if (g.second.exec) cudaGraphExecDestroy(g.second.exec);
            kv.second->graphs.clear();
        }
}

int mg_ctx_set_fp32_smoother(mg_ctx *ctx, int choice)
{
    if (!ctx) return MG_ERR_ARG;
    if (choice < -1 || choice > stream_variants())
        return set_err(ctx, MG_ERR_ARG, "fp32 smoother choice %d not in -1 .. %d", choice, stream_variants());
    ctx->fp32_smoother = choice;
    reset_fp32_tuning(ctx);
    return MG_OK;
}

int mg_ctx_set_fp32_smoother_shape(mg_ctx *ctx, int n, int bx, int zc)
{
    if (!ctx) return MG_ERR_ARG;
    if (bx == 0) {
        ctx->fp32_shape.erase(n);
    } else {
        if (n < 8 || (bx != 8 && bx != 16 && bx != 32 && bx != 64) || 4 * bx > n / 2 || zc < 1 || zc > n)
            return set_err(ctx, MG_ERR_ARG, "bad fp32 smoother shape n=%d bx=%d zc=%d", n, bx, zc);
        ctx->fp32_shape[n] = {bx, zc};
    }
    reset_fp32_tuning(ctx);
    return MG_OK;
}

long long mg_ctx_workspace_bytes(const mg_ctx *ctx)
{
    if (!ctx) return 0;
    long long b = 0;
    for (auto &p : ctx->p64) b += (long long)p.second->bytes;
    for (auto &p : ctx->p32) b += (long long)p.second->bytes;
    for (auto &p : ctx->p64c) b += (long long)p.second->bytes;
    for (auto &p : ctx->p32c) b += (long long)p.second->bytes;
    for (int q = 0; q < mg_ctx::NSTAGE; ++q) b += (long long)ctx->stage_bytes[q];
    return b;
}

int mg_solve_dgp(mg_ctx *ctx, int count, const mg_instance *inst, const mg_opts *opts, mg_stats *stats)
{
    if (!ctx) return MG_ERR_ARG;
    if (count < 1 || !inst) return set_err(ctx, MG_ERR_ARG, "count must be >= 1 and inst non-NULL");
    mg_opts o;
    if (opts)
        o = *opts;
    else
        mg_opts_default(&o);
    int rc = check_opts(ctx, o);
    if (rc) return rc;
    for (int q = 0; q < count; ++q) {
        const mg_instance &I = inst[q];
        if (!I.delta || !I.phi) return set_err(ctx, MG_ERR_ARG, "instance %d: null delta/phi", q);
        if (!valid_ng(I.g.ng)) return set_err(ctx, MG_ERR_ARG, "instance %d: ng = %d is not 2^k or 3*2^k in [8, 1536]", q, I.g.ng);
        if (!(I.g.a > 0) || !(I.g.omega_m > 0) || !(I.p.rc_h0 > 0))
            return set_err(ctx, MG_ERR_ARG, "instance %d: a, omega_m and rc_h0 must be > 0", q);
    }
    int worst = MG_OK;
    // the batched form: MIXED precision, several instances, device arrays
    bool batched = count > 1 && o.precision == MG_PREC_MIXED && (o.pre + o.post) % 2 == 0;
    for (int q = 0; batched && q < count; ++q)
        batched = is_device_ptr(inst[q].delta) && is_device_ptr(inst[q].phi);
    if (batched) {
        try {
            enter(ctx);
            worst = solve_batch(ctx, count, inst, o, stats);
            leave(ctx);
        } catch (CudaFail &f) {
            return f.code;
        }
        return worst;
    }
    try {
        enter(ctx);
        for (int q = 0; q < count; ++q) {
            const mg_instance &I = inst[q];
            const double a = I.g.a, om = I.g.omega_m, rch = I.p.rc_h0;
            const double beta = beta_dgp(a, om, rch);
            const double alpha = 3.0 * beta * a * a / (rch * rch);
            ModelDesc md{0, alpha, 0, 0.0, 0.0, (alpha / beta) * om / a, om / (a * beta)};
            rc = solve_any(ctx, I.g.ng, md, I.delta, I.phi, o, stats ? stats + q : nullptr);
            if (rc < 0) {
                leave(ctx);
                return rc;
            }
            if (rc > worst) worst = rc;
        }
        leave(ctx);
    } catch (CudaFail &f) {
        return f.code;
    }
    return worst;
}

int mg_solve_kmouflage(mg_ctx *ctx, const mg_grid *g, const mg_kmo_params *p, const mg_opts *opts,
                       const double *delta, double *phi, mg_stats *stats)
{
    if (!ctx) return MG_ERR_ARG;
    if (!g || !p || !delta || !phi) return set_err(ctx, MG_ERR_ARG, "null argument");
    if (!valid_ng(g->ng)) return set_err(ctx, MG_ERR_ARG, "ng = %d is not 2^k or 3*2^k in [8, 1536]", g->ng);
    if (p->n < 2 || p->k0 < 0 || !(g->a > 0) || !(g->box_mpch > 0) || !(p->lambda > 0))
        return set_err(ctx, MG_ERR_ARG, "bad Kmouflage parameters");
    mg_opts o;
    if (opts)
        o = *opts;
    else
        mg_opts_default(&o);
    int rc = check_opts(ctx, o);
    if (rc) return rc;
    try {
        enter(ctx);
        rc = solve_any(ctx, g->ng, kmo_desc(*g, *p), delta, phi, o, stats);
        leave(ctx);
    } catch (CudaFail &f) {
        return f.code;
    }
    return rc;
}

}  // extern "C"

// ---------------------------------------------------------------------------
// kernel-level entry points
// ---------------------------------------------------------------------------
template <typename T>
static int op_smooth_t(mg_ctx *ctx, const mg_op_params *op, int n, double h, const double *u_in, const double *s,
                       const double *f, double c, int colour, double *u_out)
{
    Pyramid<T> &P = *get_pyramid<T>(ctx, n, false);
    ModelDesc md{op->model, op->alpha, op->nkmo, op->gamma, op->bterm, 1.0, 1.0};
    upload_op(ctx, P, md);
    cudaStream_t st = ctx->stream;
    LevArrays<T> L = P.L[0];
    L.h = h;
    T *u[2] = {L.U(0), L.U(1)};
    launch_split<T>(u_in, n, u, 1.0, nullptr, st);
    launch_split<T>(s, n, L.s, 1.0, nullptr, st);
    if (f) {
        launch_split<T>(f, n, L.fbuf, 1.0, nullptr, st);
        L.f[0] = L.fbuf[0];
        L.f[1] = L.fbuf[1];
    } else {
        L.f[0] = L.f[1] = nullptr;
    }
    LevScal hs{};
    hs.c = c;
    hs.cf32 = (float)(-c);
    memcpy(ctx->hpin, &hs, sizeof hs);
    MG_CK(cudaMemcpyAsync(L.sc, ctx->hpin, sizeof hs, cudaMemcpyHostToDevice, st));
    launch_smooth<T>(L, &L, P.opT, colour, st);
    T *o2[2] = {L.U(0), L.U(1)};
    launch_merge<T>(o2, n, u_out, nullptr, st);
    MG_CK(cudaStreamSynchronize(st));
    return MG_OK;
}

// FP32 correction-form half-sweep (the inner smoother of MG_PREC_MIXED)
static int op_smooth_corr_t(mg_ctx *ctx, const mg_op_params *op, int n, double h, const double *e_in,
                            const double *base, const double *s, const double *f, double c, int colour,
                            double *e_out)
{
    Pyramid<float> &P = *get_pyramid<float>(ctx, n, true);
    ModelDesc md{op->model, op->alpha, op->nkmo, op->gamma, op->bterm, 1.0, 1.0};
    upload_op(ctx, P, md);
    cudaStream_t st = ctx->stream;
    LevArrays<float> L = P.L[0];
    L.h = h;
    float *u[2] = {L.U(0), L.U(1)};
    launch_split<float>(e_in, n, u, 1.0, nullptr, st);
    launch_split<float>(base, n, L.base, 1.0, nullptr, st);
    launch_split<float>(s, n, L.s, 1.0, nullptr, st);
    if (f) {
        launch_split<float>(f, n, L.fbuf, 1.0, nullptr, st);
        L.f[0] = L.fbuf[0];
        L.f[1] = L.fbuf[1];
    } else {
        L.f[0] = L.f[1] = nullptr;
    }
    LevScal hs{};
    hs.c = c;
    hs.cf32 = (float)(-c);
    memcpy(ctx->hpin, &hs, sizeof hs);
    MG_CK(cudaMemcpyAsync(L.sc, ctx->hpin, sizeof hs, cudaMemcpyHostToDevice, st));
    launch_smooth<float>(L, &L, P.opT, colour, st);
    float *o2[2] = {L.U(0), L.U(1)};
    launch_merge<float>(o2, n, e_out, nullptr, st);
    MG_CK(cudaStreamSynchronize(st));
    return MG_OK;
}

template <typename T>
static int op_resid_restrict_t(mg_ctx *ctx, const mg_op_params *op, int n, double h, const double *u,
                               const double *s, const double *f, double *Ru, double *Rd, double *c_out,
                               double *eps_out)
{
    Pyramid<T> &P = *get_pyramid<T>(ctx, n, false);
    if (P.nlev < 2) return set_err(ctx, MG_ERR_ARG, "n = %d has no coarser level", n);
    ModelDesc md{op->model, op->alpha, op->nkmo, op->gamma, op->bterm, 1.0, 1.0};
    upload_op(ctx, P, md);
    cudaStream_t st = ctx->stream;
    LevArrays<T> L = P.L[0];
    LevArrays<T> C = P.L[1];
    L.h = h;
    T *uu[2] = {L.U(0), L.U(1)};
    launch_split<T>(u, n, uu, 1.0, nullptr, st);
    launch_split<T>(s, n, L.s, 1.0, nullptr, st);
    if (f) {
        launch_split<T>(f, n, L.fbuf, 1.0, nullptr, st);
        L.f[0] = L.fbuf[0];
        L.f[1] = L.fbuf[1];
    } else {
        L.f[0] = L.f[1] = nullptr;
    }
    MG_CK(cudaMemsetAsync(P.scal, 0, sizeof(LevScal) * P.nlev, st));
    launch_resid_restrict<T>(L, C, P.opT, P.rb, st);
    LevScal hs;
    read_scal(ctx, L.sc, &hs);
    // the residual norm (with the compatibility constant the restriction
    // pass set) from the norm pass: the restriction pass of the V-cycle does
    // not sum d^2
    double eps2 = hs.eps2;
    if (eps_out) {
        launch_resid_norm<T>(L, P.opT, P.rb, st);
        LevScal hn;
        read_scal(ctx, L.sc, &hn);
        eps2 = hn.eps2;
    }
    T *ru[2] = {C.U(0), C.U(1)};
    launch_merge<T>(ru, n / 2, Ru, nullptr, st);
    ctx->hpin[0] = -hs.dc;
    MG_CK(cudaMemcpyAsync(ctx->dscratch, ctx->hpin, sizeof(double), cudaMemcpyHostToDevice, st));
    launch_merge<T>(C.fbuf, n / 2, Rd, ctx->dscratch, st);
    MG_CK(cudaStreamSynchronize(st));
    if (c_out) *c_out = hs.c;
    if (eps_out) *eps_out = std::sqrt(std::fmax(eps2, 0.0));
    return MG_OK;
}

template <typename T>
static int op_coarse_source_t(mg_ctx *ctx, const mg_op_params *op, int n, double h, const double *Ru,
                              const double *Rd, const double *s, double *f_out, double *c_out)
{
    Pyramid<T> &P = *get_pyramid<T>(ctx, n, false);
    ModelDesc md{op->model, op->alpha, op->nkmo, op->gamma, op->bterm, 1.0, 1.0};
    upload_op(ctx, P, md);
    cudaStream_t st = ctx->stream;
    LevArrays<T> C = P.L[0];
    C.h = h;
    C.f[0] = C.fbuf[0];
    C.f[1] = C.fbuf[1];
    launch_split<T>(Ru, n, C.ur, 1.0, nullptr, st);
    launch_split<T>(Rd, n, C.fbuf, 1.0, nullptr, st);
    launch_split<T>(s, n, C.s, 1.0, nullptr, st);
    MG_CK(cudaMemsetAsync(P.scal, 0, sizeof(LevScal) * P.nlev, st));
    // a zeroed scalar block stands in for the finer level (dc = 0)
    LevArrays<T> F = C;
    F.sc = (LevScal *)ctx->dscratch;
    MG_CK(cudaMemsetAsync(ctx->dscratch, 0, sizeof(LevScal), st));
    launch_coarse_source<T>(F, C, P.opT, P.rb, st);
    LevScal hs;
    read_scal(ctx, C.sc, &hs);
    // f = f' + fshift
    ctx->hpin[0] = -hs.fshift;
    MG_CK(cudaMemcpyAsync(ctx->dscratch + 8, ctx->hpin, sizeof(double), cudaMemcpyHostToDevice, st));
    launch_merge<T>(C.fbuf, n, f_out, ctx->dscratch + 8, st);
    MG_CK(cudaStreamSynchronize(st));
    if (c_out) *c_out = hs.c;
    return MG_OK;
}

template <typename T>
static int op_prolong_t(mg_ctx *ctx, int n, double *u_fine, const double *uc, const double *urc)
{
    Pyramid<T> &P = *get_pyramid<T>(ctx, n, false);
    if (P.nlev < 2) return set_err(ctx, MG_ERR_ARG, "n = %d has no coarser level", n);
    cudaStream_t st = ctx->stream;
    LevArrays<T> L = P.L[0], C = P.L[1];
    T *uf[2] = {L.U(0), L.U(1)};
    T *uC[2] = {C.U(0), C.U(1)};
    launch_split<T>(u_fine, n, uf, 1.0, nullptr, st);
    launch_split<T>(uc, n / 2, uC, 1.0, nullptr, st);
    launch_split<T>(urc, n / 2, C.ur, 1.0, nullptr, st);
    launch_prolong<T>(L, C, st);
    launch_merge<T>(uf, n, u_fine, nullptr, st);
    MG_CK(cudaStreamSynchronize(st));
    return MG_OK;
}

static int op_entry(mg_ctx *ctx, int n, const std::vector<const void *> &in, int precision)
{
    if (!ctx) return MG_ERR_ARG;
    if (n < 4 || n % 2) return set_err(ctx, MG_ERR_ARG, "n = %d must be even and >= 4", n);
    if (precision < 0 || precision > 1) return set_err(ctx, MG_ERR_ARG, "bad precision");
    for (auto p : in)
        if (!p) return set_err(ctx, MG_ERR_ARG, "null array");
    return MG_OK;
}

extern "C" {

int mg_op_smooth(mg_ctx *ctx, const mg_op_params *op, int precision, int n, double h, const double *u_in,
                 const double *s, const double *f, double c, int colour, double *u_out)
{
    int rc = op_entry(ctx, n, {op, u_in, s, u_out}, precision);
    if (rc) return rc;
    const size_t b = sizeof(double) * (size_t)n * n * n;
    try {
        enter(ctx);
        const double *du = (const double *)stage_in(ctx, 0, u_in, b, true);
        const double *ds = (const double *)stage_in(ctx, 1, s, b, true);
        const double *df = (const double *)stage_in(ctx, 2, f, b, true);
        double *dout = (double *)stage_in(ctx, 3, u_out, b, false);
        rc = precision ? op_smooth_t<float>(ctx, op, n, h, du, ds, df, c, colour & 1, dout)
                       : op_smooth_t<double>(ctx, op, n, h, du, ds, df, c, colour & 1, dout);
        stage_out(ctx, u_out, dout, b);
        leave(ctx);
    } catch (CudaFail &f) {
        return f.code;
    }
    return rc;
}

int mg_op_smooth_corr(mg_ctx *ctx, const mg_op_params *op, int n, double h, const double *e_in, const double *base,
                      const double *s, const double *f, double c, int colour, double *e_out)
{
    int rc = op_entry(ctx, n, {op, e_in, base, s, e_out}, 1);
    if (rc) return rc;
    const size_t b = sizeof(double) * (size_t)n * n * n;
    try {
        enter(ctx);
        const double *de = (const double *)stage_in(ctx, 0, e_in, b, true);
        const double *dbs = (const double *)stage_in(ctx, 1, base, b, true);
        const double *ds = (const double *)stage_in(ctx, 2, s, b, true);
        double *dout = (double *)stage_in(ctx, 3, e_out, b, false);
        const double *df = (const double *)stage_in(ctx, 4, f, b, true);
        rc = op_smooth_corr_t(ctx, op, n, h, de, dbs, ds, df, c, colour & 1, dout);
        stage_out(ctx, e_out, dout, b);
        leave(ctx);
    } catch (CudaFail &fl) {
        return fl.code;
    }
    return rc;
}

int mg_op_resid_restrict(mg_ctx *ctx, const mg_op_params *op, int precision, int n, double h, const double *u,
                         const double *s, const double *f, double *Ru, double *Rd, double *c_out, double *eps_out)
{
    int rc = op_entry(ctx, n, {op, u, s, Ru, Rd}, precision);
    if (rc) return rc;
    if (n < 8) return set_err(ctx, MG_ERR_ARG, "n must be >= 8");
    const size_t b = sizeof(double) * (size_t)n * n * n;
    try {
        enter(ctx);
        const double *du = (const double *)stage_in(ctx, 0, u, b, true);
        const double *ds = (const double *)stage_in(ctx, 1, s, b, true);
        const double *df = (const double *)stage_in(ctx, 2, f, b, true);
        double *dR = (double *)stage_in(ctx, 3, Ru, 2 * b / 8, false);
        double *dRu = dR, *dRd = dR + (size_t)n * n * n / 8;
        const bool hostRu = !is_device_ptr(Ru);
        if (!hostRu) {
            dRu = Ru;
            dRd = Rd;
        }
        rc = precision ? op_resid_restrict_t<float>(ctx, op, n, h, du, ds, df, dRu, dRd, c_out, eps_out)
                       : op_resid_restrict_t<double>(ctx, op, n, h, du, ds, df, dRu, dRd, c_out, eps_out);
        if (hostRu) {
            stage_out(ctx, Ru, dRu, b / 8);
            stage_out(ctx, Rd, dRd, b / 8);
        }
        leave(ctx);
    } catch (CudaFail &f) {
        return f.code;
    }
    return rc;
}

int mg_op_coarse_source(mg_ctx *ctx, const mg_op_params *op, int precision, int n, double h, const double *Ru,
                        const double *Rd, const double *s, double *f_out, double *c_out)
{
    int rc = op_entry(ctx, n, {op, Ru, Rd, s, f_out}, precision);
    if (rc) return rc;
    const size_t b = sizeof(double) * (size_t)n * n * n;
    try {
        enter(ctx);
        const double *a = (const double *)stage_in(ctx, 0, Ru, b, true);
        const double *d = (const double *)stage_in(ctx, 1, Rd, b, true);
        const double *ds = (const double *)stage_in(ctx, 2, s, b, true);
        double *dout = (double *)stage_in(ctx, 3, f_out, b, false);
        rc = precision ? op_coarse_source_t<float>(ctx, op, n, h, a, d, ds, dout, c_out)
                       : op_coarse_source_t<double>(ctx, op, n, h, a, d, ds, dout, c_out);
        stage_out(ctx, f_out, dout, b);
        leave(ctx);
    } catch (CudaFail &f) {
        return f.code;
    }
    return rc;
}

int mg_op_prolong_add(mg_ctx *ctx, int precision, int n, double *u_fine, const double *uc, const double *urc)
{
    int rc = op_entry(ctx, n, {u_fine, uc, urc}, precision);
    if (rc) return rc;
    if (n < 8) return set_err(ctx, MG_ERR_ARG, "n must be >= 8");
    const size_t b = sizeof(double) * (size_t)n * n * n;
    try {
        enter(ctx);
        double *du = (double *)stage_in(ctx, 0, u_fine, b, true);
        const double *dc = (const double *)stage_in(ctx, 1, uc, b / 8, true);
        const double *dr = (const double *)stage_in(ctx, 2, urc, b / 8, true);
        rc = precision ? op_prolong_t<float>(ctx, n, du, dc, dr) : op_prolong_t<double>(ctx, n, du, dc, dr);
        stage_out(ctx, u_fine, du, b);
        leave(ctx);
    } catch (CudaFail &f) {
        return f.code;
    }
    return rc;
}

int mg_op_coarsest(mg_ctx *ctx, const mg_op_params *op, int n, double h, double *u, const double *s,
                   const double *f, int sweeps)
{
    int rc = op_entry(ctx, n, {op, u, s}, 0);
    if (rc) return rc;
    if (n * n * n > 512) return set_err(ctx, MG_ERR_ARG, "coarsest level must have <= 512 cells");
    if (sweeps < 1) return set_err(ctx, MG_ERR_ARG, "sweeps must be >= 1");
    const size_t b = sizeof(double) * (size_t)n * n * n;
    try {
        enter(ctx);
        double *du = (double *)stage_in(ctx, 0, u, b, true);
        const double *ds = (const double *)stage_in(ctx, 1, s, b, true);
        const double *df = (const double *)stage_in(ctx, 2, f, b, true);
        Pyramid<double> &P = *get_pyramid<double>(ctx, n, false);
        ModelDesc md{op->model, op->alpha, op->nkmo, op->gamma, op->bterm, 1.0, 1.0};
        upload_op(ctx, P, md);
        cudaStream_t st = ctx->stream;
        LevArrays<double> L = P.L[P.nlev - 1 == 0 ? 0 : 0];
        L.h = h;
        double *uu[2] = {L.U(0), L.U(1)};
        launch_split<double>(du, n, uu, 1.0, nullptr, st);
        launch_split<double>(ds, n, L.s, 1.0, nullptr, st);
        if (df) {
            launch_split<double>(df, n, L.fbuf, 1.0, nullptr, st);
            L.f[0] = L.fbuf[0];
            L.f[1] = L.fbuf[1];
        } else {
            L.f[0] = L.f[1] = nullptr;
        }
        MG_CK(cudaMemsetAsync(P.scal, 0, sizeof(LevScal) * P.nlev, st));
        launch_coarsest<double>(L, P.opD, sweeps, st);
        launch_merge<double>(uu, n, du, nullptr, st);
        MG_CK(cudaStreamSynchronize(st));
        stage_out(ctx, u, du, b);
        leave(ctx);
    } catch (CudaFail &f) {
        return f.code;
    }
    return MG_OK;
}

}  // extern "C"
