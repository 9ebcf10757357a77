// Batched ensemble of nDGP solves (many independent meshes of uneven size)
// in one persistent cooperative kernel.  Every instance runs the mixed
// precision solve of solver.cu (FP64 defect, FP32 FAS correction V-cycles
// with a frozen base field, FP64 update); the kernel walks a program of
// phases, and in each phase its blocks walk the work tiles of all instances
// still iterating (per-instance reductions are finished by the instance's
// last tile), then the whole grid synchronises.  Instances with fewer
// levels idle in the deeper phases; an instance that has converged drops
// out of the work lists.  Tile widths per level size come from a small
// autotuner (measured on the one-level smoother).
#include <cooperative_groups.h>

#include <algorithm>
#include <cmath>
#include <cstring>
#include <vector>

#include "cells.cuh"
#include "ctx.cuh"

namespace cg = cooperative_groups;

namespace mg {

constexpr int BMAXL = 16;    // levels per instance
constexpr int BMAXI = 512;   // instances per batch
constexpr int BTHREADS = 256;

struct BLev {
    float *u[2][2];
    float *s[2];
    float *f[2];
    float *ur[2];
    float *base[2];
    LevScal *sc;
    int n, half;
    double h;
    int tx;          // tile width along m (threads); 256 / tx along j
    LevK<float> K;   // the level's stencil constants (computed on the host:
                     // their FP64 divisions would cost more per tile than
                     // the FP32 stencil work at the FP64 rate of this GPU)
};

struct BInst {
    BLev lev[BMAXL];
    int nlev;
    double *u64[2];
    double *s64[2];
    LevScal *sc64;
    LevK<double> K64;    // finest-level constants (h = 1)
    DgpK64 dk64;         // folded constants of the FP64 nDGP defect (h = 1)
    OpK<float> opf;
    OpK<double> opd;
    double tol;
    double *partials;
    unsigned int *counter;
    int next_active;   // written by the defect's finaliser, read after a grid sync
    int cycles;
    int converged;
    int n_eps;
    double eps[65];
};

enum { PH_SMOOTH = 0, PH_RR = 1, PH_CS = 2, PH_COARSEST = 3, PH_PROLONG = 4 };

struct Phase {
    int type, depth, colour;
    int cur[2];    // current buffers of the two colours at `depth`
    int curc[2];   // ... at depth + 1
};

struct BatchArgs {
    BInst *inst;
    int count;
    const Phase *prog;
    int nprog;
    int inner;
    int max_cycles;
    int coarse_sweeps;
};

// ---------------------------------------------------------------------------
// work tiles
// ---------------------------------------------------------------------------
__device__ __forceinline__ int cdiv(int a, int b) { return (a + b - 1) / b; }

// tiles of an (m, j) plane of level l, times the planes
__device__ __forceinline__ int mj_tiles(const BLev &L, int planes)
{
    const int ty = BTHREADS / L.tx;
    return cdiv(L.half, L.tx) * cdiv(L.n, ty) * planes;
}

// tiles of 256 quads (four cells of a colour row per thread) over a level
// whose rows are a multiple of 4 long
__device__ __forceinline__ bool quad_level(const BLev &L) { return (L.half & 3) == 0; }
__device__ __forceinline__ int quad_tiles(const BLev &L) { return cdiv(L.n * L.n * (L.half / 4), BTHREADS); }

// smoother tiles: 256 quads of one plane, walked through SZ consecutive
// planes on the larger levels (the rows of planes i and i+1 read for plane
// i are still in L1 for plane i+1)
__device__ __forceinline__ int smooth_z(const BLev &L) { return L.n >= 128 ? 4 : 1; }
__device__ __forceinline__ int smooth_tiles(const BLev &L)
{
    return cdiv(L.n * (L.half / 4), BTHREADS) * cdiv(L.n, smooth_z(L));
}

// tiles over the coarse cells (K, J) of plane I of the level below l
__device__ __forceinline__ int coarse_tiles(const BLev &L)
{
    const int nc = L.n / 2, ty = BTHREADS / L.tx;
    return cdiv(nc, L.tx) * cdiv(nc, ty) * nc;
}

// decode tile t of an (x, y) x planes grid with tile shape tx x ty
__device__ __forceinline__ void tile_xyz(int t, int gx, int gy, int tx, int &x, int &y, int &z)
{
    const int ty = BTHREADS / tx;
    const int bx = t % gx, r = t / gx;
    const int by = r % gy;
    z = r / gy;
    x = bx * tx + (int)(threadIdx.x % tx);
    y = by * ty + (int)(threadIdx.x / tx);
}

// instance of global tile t given the per-instance prefix (in shared memory)
__device__ __forceinline__ int find_inst(const int *pref, int count, int t)
{
    int lo = 0, hi = count;   // pref[lo] <= t < pref[hi]
    while (hi - lo > 1) {
        const int mid = (lo + hi) >> 1;
        if (pref[mid] <= t)
            lo = mid;
        else
            hi = mid;
    }
    return lo;
}

// ---------------------------------------------------------------------------
// the persistent kernel
// ---------------------------------------------------------------------------
__global__ void __launch_bounds__(BTHREADS, 2) k_batch(BatchArgs A)
{
    cg::grid_group grid = cg::this_grid();
    extern __shared__ double smem[];
    __shared__ int pref[BMAXI + 1];
    __shared__ unsigned char act[BMAXI];
    const int count = A.count;

    auto load_active = [&]() {
        for (int q = threadIdx.x; q < count; q += blockDim.x) act[q] = (unsigned char)A.inst[q].next_active;
        __syncthreads();
    };
    // prefix of per-instance tile counts; ntile(q) must be uniform
    auto prefix = [&](auto ntile) {
        if (threadIdx.x == 0) {
            int s = 0;
            for (int q = 0; q < count; ++q) {
                pref[q] = s;
                s += act[q] ? ntile(q) : 0;
            }
            pref[count] = s;
        }
        __syncthreads();
        return pref[count];
    };

    // FP64 defect on level 0 of every active instance, -d into the FP32
    // source; the finaliser checks convergence
    // a defect tile covers DEF_Z consecutive (colour, plane) values of one
    // (m, j) tile: each thread sums its cells before the tile's block
    // reduction, whose FP64 shuffles would otherwise cost about half as
    // much as the defect itself
    constexpr int DEF_Z = 32;
    auto defect_tiles = [&](const BLev &L0) { return mj_tiles(L0, 1) * cdiv(2 * L0.n, DEF_Z); };
    auto defect = [&]() {
        const int total = prefix([&](int q) { return defect_tiles(A.inst[q].lev[0]); });
        for (int t = blockIdx.x; t < total; t += gridDim.x) {
            const int q = find_inst(pref, count, t);
            BInst &I = A.inst[q];
            const BLev &L0 = I.lev[0];
            const int lt = t - pref[q];
            const int gx = cdiv(L0.half, L0.tx), gy = cdiv(L0.n, BTHREADS / L0.tx);
            const int plane = gx * gy;
            int m, j, z0;
            tile_xyz(lt % plane, gx, gy, L0.tx, m, j, z0);
            const int zb = (lt / plane) * DEF_Z, ze = min(2 * L0.n, zb + DEF_Z);
            const LevK<double> &K = I.K64;
            const double c_old = I.sc64->c;
            double acc[4] = {0.0, 0.0, 0.0, 0.0};
            if (m < L0.half && j < L0.n)
                for (int z = zb; z < ze; ++z)
                    resid_cell<double, false, 0>(I.opd, K, I.u64[0], I.u64[1], I.s64[0], I.s64[1], nullptr, nullptr,
                                                 nullptr, nullptr, L0.f[0], L0.f[1], c_old, z & 1, z >> 1, j, m, acc,
                                                 &I.dk64);
            double tot[4];
            const int nt = defect_tiles(L0);
            if (tile_sum<4>(acc, I.partials, I.counter, lt, nt, tot) && threadIdx.x == 0) {
                const double cnt = (double)L0.n * L0.n * L0.n;
                const double c_new = tot[0] / cnt, dc = c_new - c_old;
                set_c(I.sc64, c_new);
                I.sc64->dc = dc;
                I.sc64->eps2 = (tot[2] + 2.0 * dc * tot[1] + cnt * dc * dc) / cnt;
                I.sc64->clamps = tot[3];
                const double eps = sqrt(fmax(I.sc64->eps2, 0.0));
                if (I.n_eps < 65) I.eps[I.n_eps++] = eps;
                const bool conv = eps <= I.tol;
                I.converged = conv ? 1 : 0;
                I.next_active = (!conv && I.cycles < A.max_cycles && isfinite(eps)) ? 1 : 0;
            }
        }
    };

    // one element-wise pass over level 0 of the active instances
    auto elem0 = [&](int what) {
        const int total = prefix([&](int q) { return (int)cdiv(A.inst[q].lev[0].n * A.inst[q].lev[0].n * (A.inst[q].lev[0].n / 2), BTHREADS); });
        for (int t = blockIdx.x; t < total; t += gridDim.x) {
            const int q = find_inst(pref, count, t);
            BInst &I = A.inst[q];
            const BLev &L0 = I.lev[0];
            const long long ncol = (long long)L0.n * L0.n * (L0.n / 2);
            const long long e = (long long)(t - pref[q]) * BTHREADS + threadIdx.x;
            if (e < ncol) {
                if (what == 0) {           // base field b = fl32(u), correction e = 0
                    L0.base[0][e] = (float)I.u64[0][e];
                    L0.base[1][e] = (float)I.u64[1][e];
                    L0.u[0][0][e] = 0.f;
                    L0.u[0][1][e] = 0.f;
                } else {                   // u += e
                    I.u64[0][e] += (double)L0.u[0][0][e];
                    I.u64[1][e] += (double)L0.u[0][1][e];
                }
            }
            if (what == 0 && t == pref[q] && threadIdx.x < I.nlev) {
                LevScal z{};
                if (threadIdx.x == 0) {
                    z.fshift = -I.sc64->dc;
                    z.cf32 = (float)z.fshift;
                }
                *I.lev[threadIdx.x].sc = z;
            }
        }
    };

    // base field pyramid: b_{d+1} = R b_d
    auto restrict_base = [&](int d) {
        const int total = prefix([&](int q) { return d + 1 < A.inst[q].nlev ? coarse_tiles(A.inst[q].lev[d]) : 0; });
        for (int t = blockIdx.x; t < total; t += gridDim.x) {
            const int q = find_inst(pref, count, t);
            const BInst &I = A.inst[q];
            const BLev &L = I.lev[d];
            const int nc = L.n / 2;
            const int gx = cdiv(nc, L.tx), gy = cdiv(nc, BTHREADS / L.tx);
            int K, J, Ii;
            tile_xyz(t - pref[q], gx, gy, L.tx, K, J, Ii);
            if (K < nc && J < nc) restrict_cell<float>(L.base[0], L.base[1], I.lev[d + 1].base[0], I.lev[d + 1].base[1], L.n, Ii, J, K);
        }
    };

    auto run_phase = [&](const Phase &P) {
        const int d = P.depth;
        if (P.type == PH_COARSEST) {
            for (int q = blockIdx.x; q < count; q += gridDim.x) {
                if (!act[q] || A.inst[q].nlev - 1 != d) continue;
                const BInst &I = A.inst[q];
                const BLev &L = I.lev[d];
                coarsest_block<float, true>(L.u[P.cur[0]][0], L.u[P.cur[1]][1], L.s[0], L.s[1], L.f[0], L.f[1], L.sc, L.n,
                                            L.h, I.opd, A.coarse_sweeps, L.base[0], L.base[1], smem);
            }
            return;
        }
        if (P.type == PH_SMOOTH) {
            const int c = P.colour;
            const int total = prefix([&](int q) {
                const BLev &L = A.inst[q].lev[d];
                return d < A.inst[q].nlev - 1 ? (quad_level(L) ? smooth_tiles(L) : mj_tiles(L, L.n)) : 0;
            });
            for (int t = blockIdx.x; t < total; t += gridDim.x) {
                const int q = find_inst(pref, count, t);
                const BInst &I = A.inst[q];
                const BLev &L = I.lev[d];
                const LevK<float> &K = L.K;
                if (quad_level(L)) {
                    // in-plane quad index (row j, quad m0 / 4 fastest), then the tile's planes
                    const int qr = L.half / 4, tpp = cdiv(L.n * qr, BTHREADS), Z = smooth_z(L);
                    const int lt = t - pref[q];
                    const int Q = (lt % tpp) * BTHREADS + (int)threadIdx.x;
                    if (Q < L.n * qr) {
                        const int m0 = 4 * (Q % qr), j = Q / qr;
                        const int i0 = (lt / tpp) * Z, i1 = min(L.n, i0 + Z);
                        for (int i = i0; i < i1; ++i)
                            smooth_quad<true, 0>(I.opf, K, L.u[P.cur[c]][c], L.u[P.cur[1 - c]][1 - c],
                                                 L.u[1 - P.cur[c]][c], L.s[c], L.f[c], L.sc->cf32, c, L.base[c],
                                                 L.base[1 - c], i, j, m0);
                    }
                    continue;
                }
                const int gx = cdiv(L.half, L.tx), gy = cdiv(L.n, BTHREADS / L.tx);
                int m, j, i;
                tile_xyz(t - pref[q], gx, gy, L.tx, m, j, i);
                if (m < L.half && j < L.n)
                    smooth_cell<float, true>(I.opf, K, L.u[P.cur[c]][c], L.u[P.cur[1 - c]][1 - c], L.u[1 - P.cur[c]][c],
                                             L.s[c], L.f[c], L.sc->cf32, c, L.base[c], L.base[1 - c], i, j, m);
            }
            return;
        }
        if (P.type == PH_RR) {
            auto rr_tiles = [&](const BLev &L) {
                const int nc = L.n / 2;
                return (nc & 3) == 0 ? cdiv(nc * nc * (nc / 4), BTHREADS) : coarse_tiles(L);
            };
            const int total = prefix([&](int q) { return d < A.inst[q].nlev - 1 ? rr_tiles(A.inst[q].lev[d]) : 0; });
            for (int t = blockIdx.x; t < total; t += gridDim.x) {
                const int q = find_inst(pref, count, t);
                BInst &I = A.inst[q];
                const BLev &L = I.lev[d];
                const BLev &C = I.lev[d + 1];
                const int nc = L.n / 2;
                const int lt = t - pref[q];
                const double c_old = L.sc->c;
                const double cshift = c_old - L.sc->fshift;
                double acc[4] = {0.0, 0.0, 0.0, 0.0};
                const LevK<float> &Kf = L.K;
                if ((nc & 3) == 0) {
                    // flat index over (I, J, K0 / 4), four coarse cells per thread
                    const int qr = nc / 4;
                    const int Q = lt * BTHREADS + (int)threadIdx.x;
                    if (Q < nc * nc * qr) {
                        const int K0 = 4 * (Q % qr), r = Q / qr;
                        rr_quad<true, 0>(I.opf, Kf, L.u[P.cur[0]][0], L.u[P.cur[1]][1], L.s[0], L.s[1], L.f[0],
                                         L.f[1], L.base[0], L.base[1], cshift, C.u[P.curc[0]][0], C.u[P.curc[1]][1],
                                         C.ur[0], C.ur[1], C.f[0], C.f[1], r / nc, r % nc, K0, acc);
                    }
                } else {
                    const int gx = cdiv(nc, L.tx), gy = cdiv(nc, BTHREADS / L.tx);
                    int K, J, Ii;
                    tile_xyz(lt, gx, gy, L.tx, K, J, Ii);
                    if (K < nc && J < nc)
                        rr_cell<float, true>(I.opf, Kf, L.u[P.cur[0]][0], L.u[P.cur[1]][1], L.s[0], L.s[1], L.f[0],
                                             L.f[1], L.base[0], L.base[1], cshift, C.u[P.curc[0]][0],
                                             C.u[P.curc[1]][1], C.ur[0], C.ur[1], C.f[0], C.f[1], Ii, J, K, acc);
                }
                double tot[4];
                if (tile_sum<4>(acc, I.partials, I.counter, lt, rr_tiles(L), tot) && threadIdx.x == 0) {
                    const double cnt = (double)L.n * L.n * L.n;
                    const double c_new = tot[0] / cnt;
                    set_c(L.sc, c_new);
                    L.sc->dc = c_new - c_old;
                }
            }
            return;
        }
        if (P.type == PH_CS) {
            const int e = d + 1;   // the coarse level
            const int total = prefix([&](int q) { return d < A.inst[q].nlev - 1 ? mj_tiles(A.inst[q].lev[e], 2 * A.inst[q].lev[e].n) : 0; });
            for (int t = blockIdx.x; t < total; t += gridDim.x) {
                const int q = find_inst(pref, count, t);
                BInst &I = A.inst[q];
                const BLev &C = I.lev[e];
                const int gx = cdiv(C.half, C.tx), gy = cdiv(C.n, BTHREADS / C.tx);
                const int lt = t - pref[q];
                int m, j, z;
                tile_xyz(lt, gx, gy, C.tx, m, j, z);
                const float dcf = (float)I.lev[d].sc->dc;
                CsAcc<float> ca;
                if (m < C.half && j < C.n) {
                    const LevK<float> &Kf = C.K;
                    cs_cell<float, true>(I.opf, Kf, C.ur[0], C.ur[1], C.s[0], C.s[1], C.f[0], C.f[1], C.base[0],
                                         C.base[1], dcf, z & 1, z >> 1, j, m, ca);
                }
                double acc[2] = {ca.sum(), (double)ca.cl};
                double tot[2];
                if (tile_sum<2>(acc, I.partials, I.counter, lt, mj_tiles(C, 2 * C.n), tot) && threadIdx.x == 0) {
                    const double c = tot[0] / ((double)C.n * C.n * C.n);
                    set_c_fshift(C.sc, c, c);
                    C.sc->dc = 0.0;
                }
            }
            return;
        }
        // PH_PROLONG: level d += P(level d+1)
        const int total = prefix([&](int q) {
            const BLev &L = A.inst[q].lev[d];
            return d < A.inst[q].nlev - 1 ? (quad_level(L) ? 2 * quad_tiles(L) : mj_tiles(L, 2 * L.n)) : 0;
        });
        for (int t = blockIdx.x; t < total; t += gridDim.x) {
            const int q = find_inst(pref, count, t);
            const BInst &I = A.inst[q];
            const BLev &L = I.lev[d];
            const BLev &C = I.lev[d + 1];
            if (quad_level(L)) {
                // flat quad index over (colour, i, j, m0 / 4)
                const int qr = L.half / 4;
                const int Q = (t - pref[q]) * BTHREADS + (int)threadIdx.x;
                const int per = L.n * L.n * qr;
                if (Q < 2 * per) {
                    const int col = Q / per, rem = Q % per, r = rem / qr;
                    prolong_quad(L.u[P.cur[0]][0], L.u[P.cur[1]][1], C.u[P.curc[0]][0], C.u[P.curc[1]][1], C.ur[0],
                                 C.ur[1], L.n, col, r / L.n, r % L.n, 4 * (rem % qr));
                }
                continue;
            }
            const int gx = cdiv(L.half, L.tx), gy = cdiv(L.n, BTHREADS / L.tx);
            int m, j, z;
            tile_xyz(t - pref[q], gx, gy, L.tx, m, j, z);
            if (m < L.half && j < L.n)
                prolong_cell<float>(L.u[P.cur[0]][0], L.u[P.cur[1]][1], C.u[P.curc[0]][0], C.u[P.curc[1]][1], C.ur[0],
                                    C.ur[1], L.n, z & 1, z >> 1, j, m);
        }
    };

    int maxl = 0;
    for (int q = 0; q < count; ++q) maxl = max(maxl, A.inst[q].nlev);

    // initial defect (all instances start active).  Every block reads the
    // flags before any finaliser of the following phase may rewrite them.
    load_active();
    grid.sync();
    defect();
    grid.sync();
    while (true) {
        load_active();
        int any = 0;
        for (int q = 0; q < count; ++q) any |= act[q];
        if (!any) break;
        elem0(0);
        grid.sync();
        for (int d = 0; d + 1 < maxl; ++d) {
            restrict_base(d);
            grid.sync();
        }
        for (int k = 0; k < A.inner; ++k) {
            for (int ph = 0; ph < A.nprog; ++ph) {
                run_phase(A.prog[ph]);
                grid.sync();
            }
        }
        if (blockIdx.x == 0)
            for (int q = threadIdx.x; q < count; q += blockDim.x)
                if (act[q]) A.inst[q].cycles += A.inner;
        elem0(1);
        grid.sync();
        defect();
        grid.sync();
    }
}

// ---------------------------------------------------------------------------
// host side
// ---------------------------------------------------------------------------
static void gen_cycle(std::vector<Phase> &prog, int d, int maxl, int pre, int post, std::vector<int> &cur)
{
    auto mk = [&](int type, int colour) {
        Phase p{};
        p.type = type;
        p.depth = d;
        p.colour = colour;
        p.cur[0] = cur[2 * d];
        p.cur[1] = cur[2 * d + 1];
        p.curc[0] = d + 1 < maxl ? cur[2 * (d + 1)] : 0;
        p.curc[1] = d + 1 < maxl ? cur[2 * (d + 1) + 1] : 0;
        prog.push_back(p);
    };
    auto smooth = [&]() {
        for (int c = 0; c < 2; ++c) {
            mk(PH_SMOOTH, c);
            cur[2 * d + c] ^= 1;
        }
    };
    for (int q = 0; q < pre; ++q) smooth();
    mk(PH_RR, 0);
    mk(PH_CS, 0);
    {
        Phase p{};
        p.type = PH_COARSEST;
        p.depth = d + 1;
        p.cur[0] = cur[2 * (d + 1)];
        p.cur[1] = cur[2 * (d + 1) + 1];
        prog.push_back(p);
    }
    if (d + 2 < maxl) gen_cycle(prog, d + 1, maxl, pre, post, cur);
    mk(PH_PROLONG, 0);
    for (int q = 0; q < post; ++q) smooth();
}

struct BatchWork {
    std::vector<int> sizes;
    std::vector<std::vector<int>> tx;   // tile width per instance and level
    std::vector<Pyramid<double> *> p64;
    std::vector<Pyramid<float> *> p32;
    BInst *d_inst = nullptr;
    Phase *d_prog = nullptr;
    size_t prog_cap = 0;
    double *partials = nullptr;
    unsigned int *counters = nullptr;
};

template <typename T>
Pyramid<T> *alloc_pyramid(mg_ctx *ctx, int n, bool correction);
template <typename T>
void release_pyramid(Pyramid<T> *P);

void batch_free(mg_ctx *ctx)
{
    BatchWork *w = ctx->batch;
    if (!w) return;
    for (auto *p : w->p64) release_pyramid(p);
    for (auto *p : w->p32) release_pyramid(p);
    if (w->d_inst) cudaFree(w->d_inst);
    if (w->d_prog) cudaFree(w->d_prog);
    if (w->partials) cudaFree(w->partials);
    if (w->counters) cudaFree(w->counters);
    delete w;
    ctx->batch = nullptr;
}

// Autotuner: tile width per level size, the fastest of 8, 16, 32, 64 threads
// along m for the FP32 correction smoother on a zeroed level of that size
// (CUDA events, best of 3 after a warm-up), measured once per size and
// context.  The batched kernel uses the width for every stencil phase on
// levels of that size.
static int tuned_tile_width(mg_ctx *ctx, Pyramid<float> &P, int level)
{
    const LevArrays<float> &L = P.L[level];
    auto it = ctx->tuned_tx.find(L.n);
    if (it != ctx->tuned_tx.end()) return it->second;
    cudaStream_t s = ctx->stream;
    static thread_local OpK<float> op;
    op = make_opk<float>(0, 1.0, 0, 0.0, 0.0);
    MG_CK(cudaMemcpyAsync(P.opT, &op, sizeof op, cudaMemcpyHostToDevice, s));
    int best = 32;
    float best_ms = 1e30f;
    for (int tx : {8, 16, 32, 64}) {
        if (tx > 2 * L.half && tx > 8) continue;
        launch_smooth_shape<float>(L, P.opT, 0, tx, s);
        float t = 1e30f;
        for (int r = 0; r < 3; ++r) {
            MG_CK(cudaEventRecord(ctx->t0, s));
            launch_smooth_shape<float>(L, P.opT, r & 1, tx, s);
            MG_CK(cudaEventRecord(ctx->t1, s));
            MG_CK(cudaEventSynchronize(ctx->t1));
            float ms = 0.f;
            MG_CK(cudaEventElapsedTime(&ms, ctx->t0, ctx->t1));
            t = std::min(t, ms);
        }
        if (t < best_ms) {
            best_ms = t;
            best = tx;
        }
    }
    ctx->tuned_tx[L.n] = best;
    return best;
}

// most reduction tiles any phase of an instance uses (with its tile widths)
static size_t reduction_tiles(const Pyramid<float> &P, const std::vector<int> &tx)
{
    size_t m = 1;
    for (int l = 0; l < P.nlev; ++l) {
        const int n = P.L[l].n, half = n / 2, ty = BTHREADS / tx[l], nc = n / 2;
        m = std::max(m, (size_t)((half + tx[l] - 1) / tx[l]) * ((n + ty - 1) / ty) * 2 * n);
        m = std::max(m, (size_t)((nc + tx[l] - 1) / tx[l]) * ((nc + ty - 1) / ty) * nc);
    }
    return m;
}

int solve_batch(mg_ctx *ctx, int count, const mg_instance *inst, const mg_opts &o, mg_stats *stats)
{
    if (count > BMAXI) return set_err(ctx, MG_ERR_ARG, "batched solve: at most %d instances", BMAXI);
    if ((o.pre + o.post) % 2) return set_err(ctx, MG_ERR_ARG, "batched solve needs pre + post even");
    cudaStream_t s = ctx->stream;
    std::vector<int> sizes(count);
    for (int q = 0; q < count; ++q) sizes[q] = inst[q].g.ng;
    BatchWork *w = ctx->batch;
    if (!w || w->sizes != sizes) {
        MG_CK(cudaStreamSynchronize(s));
        batch_free(ctx);
        w = new BatchWork();
        ctx->batch = w;
        w->sizes = sizes;
        size_t cap = 1;
        for (int q = 0; q < count; ++q) {
            w->p64.push_back(alloc_pyramid<double>(ctx, sizes[q], false));
            w->p32.push_back(alloc_pyramid<float>(ctx, sizes[q], true));
            Pyramid<float> &P32 = *w->p32.back();
            MG_CK(cudaMemsetAsync(P32.block, 0, P32.block_bytes, s));
            std::vector<int> tx(P32.nlev);
            for (int l = 0; l < P32.nlev; ++l) tx[l] = tuned_tile_width(ctx, P32, l);
            w->tx.push_back(tx);
            cap = std::max(cap, reduction_tiles(P32, tx));
        }
        MG_CK(cudaMalloc(&w->d_inst, sizeof(BInst) * count));
        MG_CK(cudaMalloc(&w->partials, sizeof(double) * cap * 4 * count));
        MG_CK(cudaMalloc(&w->counters, sizeof(unsigned int) * 32 * count));
        MG_CK(cudaMemset(w->counters, 0, sizeof(unsigned int) * 32 * count));
        w->prog_cap = 0;
        ctx->batch_partial_cap = cap;
    }
    // per-instance source prep (one-level launches), as in the mixed solve
    std::vector<BInst> hI(count);
    std::vector<const double *> dl(count);
    std::vector<double *> ph(count);
    int maxl = 0;
    for (int q = 0; q < count; ++q) {
        const mg_instance &In = inst[q];
        const int n = In.g.ng;
        const double a = In.g.a, om = In.g.omega_m, rc = In.p.rc_h0;
        const double orc = 1.0 / (4.0 * rc * rc), oma = om / (a * a * a), ol = 1.0 - om;
        const double beta = 1.0 + (oma + 2.0 * ol) / (2.0 * std::sqrt(orc * (oma + ol)));
        const double alpha = 3.0 * beta * a * a / (rc * rc);
        Pyramid<double> &P64 = *w->p64[q];
        Pyramid<float> &P32 = *w->p32[q];
        dl[q] = In.delta;
        ph[q] = In.phi;
        MG_CK(cudaMemsetAsync(P64.scal, 0, sizeof(LevScal) * P64.nlev, s));
        MG_CK(cudaMemsetAsync(P32.scal, 0, sizeof(LevScal) * P32.nlev, s));
        LevScal *s0 = P64.scal;
        LevArrays<double> &U64 = P64.L[0];
        LevArrays<float> &E0 = P32.L[0];
        const long long cnt = (long long)n * n * n;
        launch_mean_nat(In.delta, cnt, &s0->mean, P64.rb, s);
        launch_split<double>(In.delta, n, U64.s, (alpha / beta) * om / a, &s0->mean, s);
        launch_rms_nat(In.delta, cnt, om / (a * beta), &s0->mean, &s0->aux, P64.rb, s);
        launch_convert<float, double>(E0.s, U64.s, U64.ncol, s);
        for (int l = 0; l + 1 < P32.nlev; ++l) launch_restrict_plain<float>(P32.L[l].s, P32.L[l].n, P32.L[l + 1].s, s);
        double *Uu[2] = {U64.U(0), U64.U(1)};
        if (o.warm_start) {
            launch_split<double>(In.phi, n, Uu, 1.0, nullptr, s);
        } else {
            MG_CK(cudaMemsetAsync(Uu[0], 0, sizeof(double) * U64.ncol, s));
            MG_CK(cudaMemsetAsync(Uu[1], 0, sizeof(double) * U64.ncol, s));
        }
        BInst &B = hI[q];
        memset(&B, 0, sizeof B);
        B.nlev = P32.nlev;
        maxl = std::max(maxl, B.nlev);
        for (int l = 0; l < P32.nlev; ++l) {
            const LevArrays<float> &L = P32.L[l];
            BLev &bl = B.lev[l];
            for (int b = 0; b < 2; ++b)
                for (int c = 0; c < 2; ++c) bl.u[b][c] = L.u[b][c];
            for (int c = 0; c < 2; ++c) {
                bl.s[c] = L.s[c];
                bl.f[c] = L.fbuf[c];
                bl.ur[c] = L.ur[c];
                bl.base[c] = L.base[c];
            }
            bl.sc = L.sc;
            bl.n = L.n;
            bl.half = L.half;
            bl.h = L.h;
            bl.tx = w->tx[q][l];
            bl.K = make_levk<float>(L.n, L.h);
        }
        B.K64 = make_levk<double>(n, 1.0);
        B.u64[0] = Uu[0];
        B.u64[1] = Uu[1];
        B.s64[0] = U64.s[0];
        B.s64[1] = U64.s[1];
        B.sc64 = s0;
        B.opf = make_opk<float>(0, alpha, 0, 0.0, 0.0);
        B.opd = make_opk<double>(0, alpha, 0, 0.0, 0.0);
        B.dk64 = make_dgpk64(1.0);
        B.partials = w->partials + (size_t)q * ctx->batch_partial_cap * 4;
        B.counter = w->counters + 32 * q;
        B.next_active = 1;
    }
    // eps_ref of every instance -> tolerance
    MG_CK(cudaStreamSynchronize(s));
    for (int q = 0; q < count; ++q) {
        LevScal h;
        MG_CK(cudaMemcpy(&h, w->p64[q]->scal, sizeof h, cudaMemcpyDeviceToHost));
        hI[q].tol = o.rtol * h.aux + o.atol;
        if (stats) {
            memset(&stats[q], 0, sizeof(mg_stats));
            stats[q].eps_ref = h.aux;
        }
    }
    // program of one batched V-cycle
    std::vector<Phase> prog;
    std::vector<int> cur(2 * maxl, 0);
    gen_cycle(prog, 0, maxl, o.pre, o.post, cur);
    for (int v : cur)
        if (v) return set_err(ctx, MG_ERR_ARG, "batched cycle does not return to its buffer state");
    if (prog.size() > w->prog_cap) {
        if (w->d_prog) MG_CK(cudaFree(w->d_prog));
        MG_CK(cudaMalloc(&w->d_prog, sizeof(Phase) * prog.size()));
        w->prog_cap = prog.size();
    }
    MG_CK(cudaMemcpyAsync(w->d_prog, prog.data(), sizeof(Phase) * prog.size(), cudaMemcpyHostToDevice, s));
    MG_CK(cudaMemcpyAsync(w->d_inst, hI.data(), sizeof(BInst) * count, cudaMemcpyHostToDevice, s));
    BatchArgs A{w->d_inst, count, w->d_prog, (int)prog.size(), o.inner_cycles > 0 ? o.inner_cycles : 4, o.max_cycles,
                o.coarse_sweeps};
    int dev = 0, sms = 0, per_sm = 0;
    MG_CK(cudaGetDevice(&dev));
    MG_CK(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev));
    const size_t smem = sizeof(double) * 5 * 8 * 8 * 8;
    MG_CK(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_batch, BTHREADS, smem));
    if (per_sm < 1) return set_err(ctx, MG_ERR_CUDA, "batched kernel cannot be resident");
    const int blocks = sms * per_sm;
    void *kargs[] = {&A};
    MG_CK(cudaEventRecord(ctx->t0, s));
    if (o.use_graph) {
        cudaGraph_t g = nullptr;
        cudaGraphExec_t ge = nullptr;
        MG_CK(cudaStreamBeginCapture(s, cudaStreamCaptureModeThreadLocal));
        cudaError_t le = cudaLaunchCooperativeKernel((void *)k_batch, dim3(blocks), dim3(BTHREADS), kargs, smem, s);
        cudaError_t ce = cudaStreamEndCapture(s, &g);
        MG_CK(le);
        MG_CK(ce);
        MG_CK(cudaGraphInstantiate(&ge, g, 0));
        MG_CK(cudaGraphLaunch(ge, s));
        MG_CK(cudaStreamSynchronize(s));
        cudaGraphExecDestroy(ge);
        cudaGraphDestroy(g);
    } else {
        MG_CK(cudaLaunchCooperativeKernel((void *)k_batch, dim3(blocks), dim3(BTHREADS), kargs, smem, s));
    }
    MG_CK(cudaEventRecord(ctx->t1, s));
    MG_CK(cudaMemcpyAsync(hI.data(), w->d_inst, sizeof(BInst) * count, cudaMemcpyDeviceToHost, s));
    // gauge and natural layout
    for (int q = 0; q < count; ++q) {
        Pyramid<double> &P64 = *w->p64[q];
        double *Uu[2] = {P64.L[0].U(0), P64.L[0].U(1)};
        launch_mean_split<double>(Uu, P64.L[0].ncol, &P64.scal[0].mean, P64.rb, s);
        launch_merge<double>(Uu, sizes[q], ph[q], &P64.scal[0].mean, s);
    }
    MG_CK(cudaStreamSynchronize(s));
    float ms = 0.f;
    MG_CK(cudaEventElapsedTime(&ms, ctx->t0, ctx->t1));
    int worst = MG_OK;
    for (int q = 0; q < count; ++q) {
        const BInst &B = hI[q];
        LevScal h;
        MG_CK(cudaMemcpy(&h, w->p64[q]->scal, sizeof h, cudaMemcpyDeviceToHost));
        const int rc = B.converged ? MG_OK : MG_WARN_NOT_CONVERGED;
        if (!std::isfinite(B.eps[std::max(0, B.n_eps - 1)])) worst = MG_ERR_NONFINITE;
        if (rc > worst && worst >= 0) worst = rc;
        if (stats) {
            mg_stats &S = stats[q];
            S.cycles = B.cycles;
            S.status = rc;
            S.n_eps = B.n_eps;
            for (int e = 0; e < B.n_eps && e < 65; ++e) S.eps[e] = B.eps[e];
            S.c_final = h.c;
            S.mean_shift = h.mean;
            S.sqrt_clamps = (long long)h.clamps;
            S.ms = ms;
            long long per = 0;
            for (int l = 0; l < B.nlev; ++l) {
                const long long cells = (long long)B.lev[l].n * B.lev[l].n * B.lev[l].n;
                per += (l == B.nlev - 1 ? (long long)o.coarse_sweeps : (long long)(o.pre + o.post)) * cells;
            }
            S.cell_updates = per * B.cycles;
            // source prep and gauge fix per instance; the persistent kernel
            // is counted with the first instance
            S.kernel_launches = 5 + (B.nlev - 1) + (o.warm_start ? 1 : 0) + 2 + (q == 0 ? 1 : 0);
        }
    }
    if (worst == MG_WARN_NOT_CONVERGED) set_err(ctx, worst, "batched solve: some instances did not converge");
    if (worst == MG_ERR_NONFINITE) set_err(ctx, worst, "batched solve: non-finite residual");
    return worst;
}

}  // namespace mg
