// Host-side context of libmgglam.so: streams, workspace pyramids, staging
// buffers and error reporting shared by the solver and particle-mesh units.
#pragma once
#include <cuda_runtime.h>

#include <cstdio>
#include <map>
#include <string>
#include <tuple>
#include <vector>

#include "../../include/mgglam.h"
#include "kernels.cuh"

namespace mg {

// A CUDA error inside the library is reported by returning MG_ERR_CUDA with
// the failing call recorded in ctx->err.
struct CudaFail {
    int code;
};

#define MG_CK(call)                                                                                   \
    do {                                                                                              \
        cudaError_t e_ = (call);                                                                      \
        if (e_ != cudaSuccess) {                                                                      \
            ::mg::fail_cuda(ctx, e_, #call, __FILE__, __LINE__);                                     \
            throw ::mg::CudaFail{e_ == cudaErrorMemoryAllocation ? MG_ERR_OOM : MG_ERR_CUDA};       \
        }                                                                                             \
    } while (0)

struct CycleKey {
    std::vector<int> state;  // cur[] of every level before the cycle
    int pre, post, cycle, coarse_sweeps, nlev, prof, norm;
    int model;               // the kernels are specialised on the operator
    bool operator<(const CycleKey &o) const
    {
        return std::tie(state, pre, post, cycle, coarse_sweeps, nlev, prof, norm, model) <
               std::tie(o.state, o.pre, o.post, o.cycle, o.coarse_sweeps, o.nlev, o.prof, o.norm, o.model);
    }
};

struct GraphEntry {
    cudaGraphExec_t exec = nullptr;
    std::vector<int> post_state;
    int nprof = 0;  // profiled smoother launches recorded in the graph
};

// One multigrid level pyramid for a finest size n0 in storage type T.
template <typename T>
struct Pyramid {
    int n0 = 0, nlev = 0;
    bool correction = false;           // arrays for the MIXED correction form
    std::vector<LevArrays<T>> L;
    LevScal *scal = nullptr;           // device [nlev]
    OpK<T> *opT = nullptr;             // device operator (storage precision)
    OpK<double> *opD = nullptr;        // device operator (FP64, coarsest)
    RedBuf rb{};
    void *block = nullptr;             // one allocation carved into the arrays
    size_t block_bytes = 0;
    size_t bytes = 0;
    std::map<CycleKey, GraphEntry> graphs;

    std::vector<int> state() const
    {
        std::vector<int> s;
        for (auto &l : L) {
            s.push_back(l.cur[0]);
            s.push_back(l.cur[1]);
        }
        return s;
    }
    void set_state(const std::vector<int> &s)
    {
        for (size_t q = 0; q < L.size(); ++q) {
            L[q].cur[0] = s[2 * q];
            L[q].cur[1] = s[2 * q + 1];
        }
    }
};

struct PmWork;     // particle-mesh workspace (pm.cu)
struct BatchWork;  // batched-ensemble workspace (batch.cu)
struct DpmWork;    // differentiable particle-mesh workspace (dpm.cu)

struct ModelDesc {
    int model;         // 0 nDGP, 1 Kmouflage
    double alpha;
    int nkmo;
    double gamma, bterm;
    double s_coef;     // s = s_coef (delta - <delta>)
    double eref_coef;  // eps_ref = rms(eref_coef (delta - <delta>))
};


}  // namespace mg

struct mg_ctx {
    int device = 0;
    cudaStream_t stream = nullptr;   // internal stream (all work, captures)
    cudaStream_t ustream = nullptr;  // caller's stream (ordered around each call)
    cudaEvent_t ev_in = nullptr, ev_out = nullptr, t0 = nullptr, t1 = nullptr;
    std::string err;
    std::map<int, mg::Pyramid<double> *> p64;
    std::map<int, mg::Pyramid<float> *> p32;
    std::map<int, mg::Pyramid<double> *> p64c;  // correction-form pyramids
    std::map<int, mg::Pyramid<float> *> p32c;
    // staging for host pointers: grow-only device buffers
    static constexpr int NSTAGE = 6;
    void *stage[NSTAGE] = {};
    size_t stage_bytes[NSTAGE] = {};
    double *hpin = nullptr;          // pinned host scratch (64 doubles)
    double *dscratch = nullptr;      // device scratch (64 doubles)
    mg::RedBuf rb{};                 // reduction buffer for stand-alone reductions
    mg::PmWork *pm = nullptr;
    mg::BatchWork *batch = nullptr;
    void *adj = nullptr;             // adjoint workspace (adjoint.cu)
    mg::DpmWork *dpm = nullptr;      // differentiable PM workspace (dpm.cu)
    size_t batch_partial_cap = 0;    // reduction tiles per instance
    std::map<int, int> tuned_tx;     // autotuned tile width per level size
    // profiling of the finest-level smoother (events recorded in the graphs)
    int prof_on = 0;
    int fp32_smoother = 0;           // -1 gathering kernel, 0 autotuned, k > 0 streaming variant k
    std::map<int, std::pair<int, int>> fp32_shape;  // pinned (bx, zc) of the gathering kernel per level size
    int prof_k = 0;                  // launches bracketed in the current cycle
    std::vector<cudaEvent_t> pev;    // pairs (start, stop)
};

namespace mg {

void fail_cuda(mg_ctx *ctx, cudaError_t e, const char *call, const char *file, int line);
int set_err(mg_ctx *ctx, int code, const char *fmt, ...);
bool is_device_ptr(const void *p);
// device view of a caller array: the pointer itself if it is on the device,
// else staging slot `slot` filled from the host (if copy_in).
void *stage_in(mg_ctx *ctx, int slot, const void *p, size_t bytes, bool copy_in);
void stage_out(mg_ctx *ctx, void *host, const void *dev, size_t bytes);
size_t level_count(int n);
bool valid_ng(int n);
template <typename T>
Pyramid<T> *get_pyramid(mg_ctx *ctx, int n, bool correction);
// an uncached pyramid owned by the caller (batched solves), and its release
template <typename T>
Pyramid<T> *alloc_pyramid(mg_ctx *ctx, int n, bool correction);
template <typename T>
void release_pyramid(Pyramid<T> *P);
int solve_batch(mg_ctx *ctx, int count, const mg_instance *inst, const mg_opts &o, mg_stats *stats);
void batch_free(mg_ctx *ctx);
void adj_release(mg_ctx *ctx);

// entry/exit ordering with the caller's stream
void enter(mg_ctx *ctx);
void leave(mg_ctx *ctx);

// nDGP solve on device arrays (validated options), and the CIC deposit
int solve_dgp_dev(mg_ctx *ctx, int n, double a, double om, double rc, const double *delta, double *phi,
                  const mg_opts &o, mg_stats *st);
int solve_kmo_dev(mg_ctx *ctx, const mg_grid &g, const mg_kmo_params &p, const double *delta, double *phi,
                  const mg_opts &o, mg_stats *st);
void cic_deposit_dev(mg_ctx *ctx, int ng, const float *pos, long long np, double *delta);
int check_opts(mg_ctx *ctx, const mg_opts &o);

// FFT workspace of the particle-mesh step for an n^3 mesh, and the
// Newtonian potential Lap Phi = (3/2) Omega_m a^-1 delta on device arrays
void pm_fft_setup(mg_ctx *ctx, int n);
void newton_potential_dev(mg_ctx *ctx, int n, double a, double om, const double *delta, double *out);
void poisson_dev(mg_ctx *ctx, int n, double coef, const double *rhs, double *out);
// the nDGP adjoint solve on device arrays (validated arguments)
int adjoint_dev(mg_ctx *ctx, int n, double a, double om, double Rc, const mg_opts &o, const double *dphi,
                const double *ddel, const double *dg, double *dout, double *drc, mg_stats *st);
void dpm_release(mg_ctx *ctx);

}  // namespace mg
