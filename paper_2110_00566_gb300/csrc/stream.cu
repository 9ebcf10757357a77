// Streaming FP32 four-cell smoother for the 256^3 and 512^3 levels of the
// mixed-precision solve: one colour-simultaneous half-sweep of Eq.
// nonlinear_GS_DGP (nDGP) or of the Kmouflage update, plain or in the
// correction form, with the same per-quad arithmetic as k_smooth4 (the
// stencil rows come through the SRows accessor instead of GRows), so both
// kernels give bit-identical fields.  The solver's autotuner times it
// against the gathering kernel per level and keeps the faster.
//
// Every plane of the stencil's fields (the unknown of both colours, and in
// the correction form the base field of both colours) that a block needs is
// staged in shared memory by bulk asynchronous copies (the TMA unit:
// cp.async.bulk with mbarrier completion): a slot holds rows j0-1 .. j0+TJ
// (periodically wrapped) of one plane, one copy per field, and a ring of
// slots keeps the planes ahead of the compute in flight.  The source s and
// the FAS right-hand side f are read once per cell straight from global
// memory (L2-prefetched when their plane's upper neighbour is issued, and
// loaded a plane ahead into registers).
//
// Every wait on an mbarrier is bounded: on timeout the warp records the
// failure in a device flag and leaves, after waiting (bounded) for the
// latest copy issued into each slot; the solver turns the flag into
// MG_ERR_TIMEOUT.
#include <algorithm>
#include <cstdint>

#include "cells.cuh"
#include "kernels.cuh"

namespace mg {

namespace {

constexpr long long WAIT_POLLS = 1LL << 22;

__device__ int g_stream_timeout = 0;

__device__ __forceinline__ unsigned smem_u32(const void *p) { return (unsigned)__cvta_generic_to_shared(p); }

__device__ __forceinline__ void mbar_init(unsigned long long *bar, unsigned count)
{
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(bar)), "r"(count) : "memory");
}

__device__ __forceinline__ void mbar_arrive_tx(unsigned long long *bar, unsigned bytes)
{
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_u32(bar)), "r"(bytes)
                 : "memory");
}

__device__ __forceinline__ bool mbar_try(unsigned long long *bar, unsigned parity)
{
    unsigned ok;
    asm volatile(
        "{\n\t.reg .pred p;\n\t"
        "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
        "selp.u32 %0, 1, 0, p;\n\t}"
        : "=r"(ok)
        : "r"(smem_u32(bar)), "r"(parity)
        : "memory");
    return ok != 0;
}

__device__ __forceinline__ bool mbar_wait(unsigned long long *bar, unsigned parity)
{
    for (long long it = 0; it < WAIT_POLLS; ++it)
        if (mbar_try(bar, parity)) return true;
    return false;
}

__device__ __forceinline__ void bulk_g2s(void *dst, const void *src, unsigned bytes, unsigned long long *bar)
{
    asm volatile(
        "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(
            smem_u32(dst)),
        "l"(src), "r"(bytes), "r"(smem_u32(bar))
        : "memory");
}

constexpr int MAXSLOT = 12;

struct StreamArgs {
    const float *f[4];     // stencil fields: updated colour, other colour (, base: updated, other)
    const float *Sc, *Fc;  // source and FAS right-hand side of the updated colour (Fc may be null)
    float *Un;             // output rows of the updated colour
    const LevScal *sc;
    LevK<float> L;
    const OpK<float> *op;
    int colour, TJ, nslot;
};

template <bool CORR>
__host__ __device__ constexpr int stencil_fields()
{
    return CORR ? 4 : 2;
}

// floats of one plane slot: rows j0-1 .. j0+TJ of every stencil field
template <bool CORR>
__host__ __device__ inline int slot_floats(int TJ, int half)
{
    return stencil_fields<CORR>() * (TJ + 2) * half;
}

// copies of plane Pl (any integer: wrapped) into one slot: rows j0-1 ..
// j0+TJ of a field are contiguous in the colour-split layout, so a field is
// one bulk copy, or two where the tile wraps around j = 0 / j = n-1.
// Issued by one full warp (lanes 0 .. NF-1), the byte count registered on
// the slot's barrier first.
template <bool CORR>
__device__ void issue_plane(const StreamArgs &A, float *slot, unsigned long long *bar, int Pl, int j0, int lane)
{
    const int n = A.L.n, half = A.L.half, TJ = A.TJ;
    const int Pw = Pl < 0 ? Pl + n : (Pl >= n ? Pl - n : Pl);
    constexpr int NF = stencil_fields<CORR>();
    const unsigned rowb = (unsigned)half * 4u;
    if (lane == 0) mbar_arrive_tx(bar, rowb * (unsigned)(NF * (TJ + 2)));
    __syncwarp();
    if (lane < NF) {
        const float *fa = lane == 0 ? A.f[0] : lane == 1 ? A.f[1] : lane == 2 ? A.f[2] : A.f[3];
        const float *pl = fa + (long long)Pw * n * half;
        float *dst = slot + lane * (TJ + 2) * half;
        if (j0 == 0) {                 // row n-1, then rows 0 .. TJ
            bulk_g2s(dst, pl + (long long)(n - 1) * half, rowb, bar);
            bulk_g2s(dst + half, pl, rowb * (unsigned)(TJ + 1), bar);
        } else if (j0 + TJ == n) {     // rows j0-1 .. n-1, then row 0
            bulk_g2s(dst, pl + (long long)(j0 - 1) * half, rowb * (unsigned)(TJ + 1), bar);
            bulk_g2s(dst + (TJ + 1) * half, pl, rowb, bar);
        } else {
            bulk_g2s(dst, pl + (long long)(j0 - 1) * half, rowb * (unsigned)(TJ + 2), bar);
        }
    }
}

// L2 prefetch of the TJ rows of s (and f) of plane Pl that the warps read
// straight from global memory (contiguous: one prefetch per array)
__device__ __forceinline__ void prefetch_sources(const StreamArgs &A, int Pl, int j0, int lane)
{
    const int n = A.L.n, half = A.L.half;
    if (lane < (A.Fc ? 2 : 1)) {
        const float *src = (lane == 0 ? A.Sc : A.Fc) + ((long long)Pl * n + j0) * half;
        asm volatile("cp.async.bulk.prefetch.L2.global [%0], %1;" ::"l"(src), "r"((unsigned)half * 4u * A.TJ)
                     : "memory");
    }
}

template <bool CORR, int MODEL, int P>
__device__ __forceinline__ float4 quad_from_slots(const OpK<float> &op, const LevK<float> &L, const float *pm,
                                                  const float *pc, const float *pp, int TJ, int jj, int m0,
                                                  const float4 &sv, const float4 &fv, float cf)
{
    const SRows re{pm, pc, pp, 0, 1, TJ, jj, m0, L.half};
    const SRows rb{pm, pc, pp, 2, 3, TJ, jj, m0, L.half};
    if (MODEL == 0) {
        Terms4 te, tb;
        terms_rows<P>(te, re);
        if (CORR) terms_rows<P>(tb, rb);
        return dgp_quad_update<CORR>(op, L, te, tb, sv, fv, cf);
    } else {
        Quad ge, gb;
        gather_rows<P>(ge, re);
        if (CORR) gather_rows<P>(gb, rb);
        return quad_all<CORR, MODEL>(op, L, ge, gb, sv, fv, cf);
    }
}

// sequence plane q of a block's share [u0, u1) of (j-tile, plane) units:
// the share is walked as runs of consecutive planes of one j-tile, and run
// (jt, ia .. ib-1) contributes planes ia-1 .. ib (ib - ia + 2 of them)
// (t: the plane's index within its run, 0 .. ib - ia + 1)
__device__ __forceinline__ void seq_plane(long long q, long long u0, long long u1, int n, int &jt, int &P, int &t)
{
    for (long long u = u0; u < u1;) {
        const int jtile = (int)(u / n), ia = (int)(u % n);
        const int ib = (int)min((long long)n, ia + (u1 - u));
        if (q < ib - ia + 2) {
            jt = jtile;
            t = (int)q;
            P = ia - 1 + t;
            return;
        }
        q -= ib - ia + 2;
        u += ib - ia;
    }
    jt = 0;
    P = 0;
    t = 0;
}

__device__ __forceinline__ long long seq_length(long long u0, long long u1, int n)
{
    long long T = 0;
    for (long long u = u0; u < u1;) {
        const int ia = (int)(u % n);
        const int ib = (int)min((long long)n, ia + (u1 - u));
        T += ib - ia + 2;
        u += ib - ia;
    }
    return T;
}

// Persistent half-sweep.  The (j-tile, plane) units of the level are split
// evenly over the blocks; a block's share is a few runs of consecutive
// planes of one j-tile.  Plane q of the block's sequence lives in ring slot
// q % nslot; its `full` barrier completes when its copies have landed.  Each
// warp updates one quad per thread per plane from the slots of planes i-1,
// i, i+1, then releases plane i-1 on the slot's release counter; the warp
// that releases last refills the slot at once with plane q + nslot.  No
// producer warp and no block-wide synchronisation inside the loop.
template <bool CORR, int MODEL, int W>
__global__ void __launch_bounds__(32 * W, 1) k_smooth4s(StreamArgs A)
{
    extern __shared__ __align__(128) float smem[];
    __shared__ unsigned long long full[MAXSLOT];
    __shared__ int relcnt[MAXSLOT];
    __shared__ long long lastq[MAXSLOT];  // latest plane issued into each slot (-1: none)
    const int n = A.L.n, half = A.L.half, TJ = A.TJ, NS = A.nslot;
    const long long U = (long long)(n / TJ) * n;
    const long long u0 = U * blockIdx.x / gridDim.x, u1 = U * (blockIdx.x + 1) / gridDim.x;
    if (u0 >= u1) return;
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int sf = slot_floats<CORR>(TJ, half);
    const long long T = seq_length(u0, u1, n);
    if (threadIdx.x == 0) {
        for (int s = 0; s < NS; ++s) {
            mbar_init(&full[s], 1);
            relcnt[s] = 0;
            lastq[s] = -1;
        }
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    __syncthreads();
    auto issue = [&](long long q) {
        int jt, P, t;
        seq_plane(q, u0, u1, n, jt, P, t);
        if (lane == 0) lastq[q % NS] = q;
        issue_plane<CORR>(A, smem + (q % NS) * sf, &full[q % NS], P, jt * TJ, lane);
        // s and f of cell plane P - 1 (updated when this plane is its upper
        // neighbour; t >= 2 means P - 1 is one of the run's cell planes)
        if (t >= 2) prefetch_sources(A, P - 1, jt * TJ, lane);
    };
    if (warp == 0)
        for (long long q = 0; q < NS && q < T; ++q) issue(q);
    // release plane q (this warp is done with it); the last warp refills the slot
    auto release = [&](long long q) {
        __syncwarp();
        int last = 0;
        if (lane == 0) {
            __threadfence_block();
            last = atomicAdd(&relcnt[q % NS], 1) == W - 1;
            if (last) relcnt[q % NS] = 0;
            __threadfence_block();
        }
        if (__shfl_sync(0xffffffffu, last, 0) && q + NS < T) {
            asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
            issue(q + NS);
        }
    };
    const float cf = smooth_cf<float>(A.sc);
    const OpK<float> op = *A.op;
    const int qrow = half / 4;
    const int jj = threadIdx.x / qrow, m0 = 4 * (threadIdx.x % qrow);
    bool failed = false;
    long long k = 0;  // sequence index of the current run's first plane
    for (long long u = u0; u < u1 && !failed;) {
        const int jt = (int)(u / n), ia = (int)(u % n);
        const int ib = (int)min((long long)n, ia + (u1 - u));
        const int j = jt * TJ + jj;
        const long long plane = (long long)n * half;
        long long idx = ((long long)ia * n + j) * half + m0;
        float4 sv = ld4(A.Sc + idx);
        float4 fv = A.Fc ? ld4(A.Fc + idx) : make_float4(0.f, 0.f, 0.f, 0.f);
        for (int i = ia; i < ib; ++i, idx += plane) {
            const long long km = k + (i - ia);
            // the next plane's s and f, in flight during this plane's update
            float4 sn = sv, fn = fv;
            if (i + 1 < ib) {
                sn = ld4(A.Sc + idx + plane);
                if (A.Fc) fn = ld4(A.Fc + idx + plane);
            }
            for (long long q = (i == ia ? km : km + 2); q <= km + 2; ++q)
                if (!mbar_wait(&full[q % NS], (unsigned)((q / NS) & 1))) failed = true;
            if (__any_sync(0xffffffffu, failed)) {
                failed = true;
                break;
            }
            const float *pm = smem + (km % NS) * sf, *pc = smem + ((km + 1) % NS) * sf,
                        *pp = smem + ((km + 2) % NS) * sf;
            const int p = (A.colour + i + j) & 1;
            const float4 out = p ? quad_from_slots<CORR, MODEL, 1>(op, A.L, pm, pc, pp, TJ, jj, m0, sv, fv, cf)
                                 : quad_from_slots<CORR, MODEL, 0>(op, A.L, pm, pc, pp, TJ, jj, m0, sv, fv, cf);
            *reinterpret_cast<float4 *>(A.Un + idx) = out;
            release(km);
            sv = sn;
            fv = fn;
        }
        if (failed) break;
        // the run's last two planes are released once it is done
        const long long kl = k + (ib - ia);
        release(kl);
        release(kl + 1);
        k = kl + 2;
        u += ib - ia;
    }
    if (failed && lane == 0) {
        atomicExch(&g_stream_timeout, 1);
        // the block must not leave with copies in flight into its shared
        // memory: wait (bounded) for the latest plane issued into each slot
        for (int s = 0; s < NS; ++s) {
            const long long q = *(volatile long long *)&lastq[s];
            if (q >= 0) mbar_wait(&full[s], (unsigned)((q / NS) & 1));
        }
    }
}

struct Variant {
    int w;         // warps per block
    int budget;    // shared memory per block (bytes) for the ring
};
constexpr Variant VARIANTS[] = {{16, 200 * 1024}, {8, 200 * 1024}};
constexpr int NVAR = sizeof(VARIANTS) / sizeof(VARIANTS[0]);

template <bool CORR, int MODEL, int W>
void set_smem_attr()
{
    cudaFuncSetAttribute(k_smooth4s<CORR, MODEL, W>, cudaFuncAttributeMaxDynamicSharedMemorySize, 200 * 1024);
}

template <bool CORR>
void setup_corr()
{
    set_smem_attr<CORR, 0, 8>();
    set_smem_attr<CORR, 0, 16>();
    set_smem_attr<CORR, 1, 8>();   // Kmouflage: 8 warps only (~210 registers a thread)
}

// persistent grid: as many blocks as fit on the GPU at once; false (nothing
// launched) when a block does not fit on an SM
template <bool CORR, int MODEL, int W>
bool launch_w(const StreamArgs &A, size_t smem, cudaStream_t st)
{
    int dev = 0, sms = 0, per_sm = 0;
    if (cudaGetDevice(&dev) != cudaSuccess ||
        cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess ||
        cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_smooth4s<CORR, MODEL, W>, 32 * W, smem) !=
            cudaSuccess ||
        per_sm < 1)
        return false;
    k_smooth4s<CORR, MODEL, W><<<sms * per_sm, 32 * W, smem, st>>>(A);
    return true;
}

}  // namespace

int stream_variants() { return NVAR; }

bool stream_eligible(const LevArrays<float> &L)
{
    return (L.n == 256 || L.n == 512) && (L.model == 0 || L.model == 1) && L.ncol < (1LL << 31);
}

void stream_setup()
{
    static bool done = false;
    if (done) return;
    done = true;
    setup_corr<true>();
    setup_corr<false>();
}

bool launch_smooth_stream(const LevArrays<float> &L, const LevK<float> &K, const OpK<float> *op, int colour, int nb,
                          int variant, cudaStream_t st)
{
    if (variant < 1 || variant > NVAR || !stream_eligible(L)) return false;
    const Variant v = VARIANTS[variant - 1];
    // Kmouflage's quad update holds ~210 registers: 8 warps at most
    if (L.model == 1 && v.w > 8) return false;
    stream_setup();
    const bool corr = L.base[0] != nullptr;
    // bulk copies need 16-byte aligned rows
    auto al = [](const void *q) { return q == nullptr || ((uintptr_t)q & 15) == 0; };
    if (!al(L.U(0)) || !al(L.U(1)) || !al(L.base[0]) || !al(L.base[1]) || !al(L.s[colour]) || !al(L.f[colour]) ||
        !al(L.u[nb][colour]))
        return false;
    StreamArgs A;
    A.f[0] = L.U(colour);
    A.f[1] = L.U(1 - colour);
    A.f[2] = corr ? L.base[colour] : nullptr;
    A.f[3] = corr ? L.base[1 - colour] : nullptr;
    A.Sc = L.s[colour];
    A.Fc = L.f[colour];
    A.Un = L.u[nb][colour];
    A.sc = L.sc;
    A.L = K;
    A.op = op;
    A.colour = colour;
    A.TJ = 4 * 32 * v.w / L.half;
    const size_t slot = sizeof(float) * (size_t)(corr ? slot_floats<true>(A.TJ, L.half) : slot_floats<false>(A.TJ, L.half));
    A.nslot = (int)std::min<size_t>(MAXSLOT, v.budget / slot);
    if (A.nslot < 4 || L.n % A.TJ != 0) return false;
    const size_t smem = slot * A.nslot;
    if (corr) {
        if (L.model == 1) return launch_w<true, 1, 8>(A, smem, st);
        return v.w == 16 ? launch_w<true, 0, 16>(A, smem, st) : launch_w<true, 0, 8>(A, smem, st);
    }
    if (L.model == 1) return launch_w<false, 1, 8>(A, smem, st);
    return v.w == 16 ? launch_w<false, 0, 16>(A, smem, st) : launch_w<false, 0, 8>(A, smem, st);
}

int stream_timeout_flag(cudaStream_t st, bool reset)
{
    int h = 0;
    if (cudaMemcpyFromSymbolAsync(&h, g_stream_timeout, sizeof(int), 0, cudaMemcpyDeviceToHost, st) != cudaSuccess)
        return -1;
    if (cudaStreamSynchronize(st) != cudaSuccess) return -1;
    if (reset && h) {
        const int z = 0;
        if (cudaMemcpyToSymbolAsync(g_stream_timeout, &z, sizeof(int), 0, cudaMemcpyHostToDevice, st) != cudaSuccess)
            return -1;
        if (cudaStreamSynchronize(st) != cudaSuccess) return -1;
    }
    return h;
}

}  // namespace mg
