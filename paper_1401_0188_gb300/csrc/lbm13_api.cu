// lbm13_api.cu -- the C ABI declared in include/lbm13.h: parameter derivation
// (Sec. 2), lattice life cycle, state transfer and kernel dispatch.
#include <algorithm>
#include <cmath>
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <string>
#include <vector>

#include <nvtx3/nvToolsExt.h>

#include "../../include/lbm13.h"
#include "lbm13_internal.h"
#include "lbm13_coef.h"
#include "lbm13_tma.h"
#include "lbm13_pair.h"

using namespace lbm13;

struct lbm13_lattice {
    int nx = 0, ny = 0, precision = 0, device = 0;
    long long pitch = 0, plane = 0;
    size_t elem = 0, state_bytes = 0, bytes_held = 0;
    lbm13_params p{};
    lbm13_boundary b{};
    lbm13_allocator alloc{};
    bool has_alloc = false;
    cudaStream_t stream = nullptr;
    void *buf[2] = {nullptr, nullptr};
    unsigned long long *bad = nullptr;  // debug builds: accesses outside the lattice
    int cur = 0;
    long long t = 0;
    double derived[LBM13_DERIVED_COUNT] = {};
    Coef<double> kd{};
    Coef<float> kf{};
    WallArgs<double> wd[4]{};
    WallArgs<float> wf[4]{};
    bool force = false;
    // CUDA graphs of kGraphSteps steps, one per starting buffer parity
    cudaStream_t cap_stream = nullptr;
    cudaGraphExec_t gexec[2] = {nullptr, nullptr};
    // host transfers of large lattices in row bands: the copies on io_stream
    // overlap the kernels of the neighbouring bands on `stream`
    cudaStream_t io_stream = nullptr;
    cudaEvent_t io_ev[2 * 8 + 1] = {};  // 2 kIoBands + 1
    // paired steps (FP32, periodic in x and y): mode (LBM13_PAIR_*), 1 once
    // the tensor maps of both buffers are made, 0 when not possible, -1 not
    // yet considered; graphs of kGraphSteps / 2 paired launches
    int pair_mode = LBM13_PAIR_AUTO;
    int pair_ok = -1;
    CUtensorMap pair_map[2];
    cudaGraphExec_t gexec2[2] = {nullptr, nullptr};
    // persistent multi-step launches: mode (LBM13_PERSISTENT_*), grid barrier
    // words (count, generation, error), grid size (0: not possible)
    int persistent = LBM13_PERSISTENT_AUTO;
    void *sync_mem = nullptr;
    int multi_grid = -1;
    // reductions
    void *red_mem = nullptr;
    ReduceBufs rb{};
    // Fourier projections: partials [proj_blocks][kProj], then kProj results
    void *proj_mem = nullptr;
    int proj_blocks = 0;
    double *out_dev = nullptr;
    int have_snap = 0;
    long long snap_t = 0;
    std::string err;
};

namespace {

thread_local std::string g_err;

const char *kVersion = "lbm13 1.0 (D2Q13 energy-conserving MRT, sm_103a)";

int fail(lbm13_t h, int code, const std::string &msg)
{
    if (h) h->err = msg;
    g_err = msg;
    return code;
}

int check_barrier_error(lbm13_t h);

int cuda_fail(lbm13_t h, cudaError_t e, const char *where)
{
    return fail(h, LBM13_ECUDA, std::string(where) + ": " + cudaGetErrorString(e));
}

#define CK(h, call)                                              \
    do {                                                         \
        cudaError_t e_ = (call);                                 \
        if (e_ != cudaSuccess) return cuda_fail((h), e_, #call); \
    } while (0)

// Synchronises the lattice's stream and reports a grid-barrier timeout of an
// earlier persistent launch (LBM13_ETIMEOUT).
#define SYNC_CHECK(h)                                     \
    do {                                                  \
        CK((h), cudaStreamSynchronize((h)->stream));      \
        const int rc_ = check_barrier_error(h);           \
        if (rc_ != LBM13_OK) return rc_;                  \
    } while (0)

// NVTX range over one entry point (a no-op unless a profiler is attached), so
// that a timeline shows steps, read-outs and plan calls by name.
struct Range {
    explicit Range(const char *name) { nvtxRangePushA(name); }
    ~Range() { nvtxRangePop(); }
    Range(const Range &) = delete;
    Range &operator=(const Range &) = delete;
};

// Keeps the lattice's device current for the duration of a call.
struct DeviceGuard {
    int prev = -1;
    bool ok = true;
    explicit DeviceGuard(int dev)
    {
        if (cudaGetDevice(&prev) != cudaSuccess) { ok = false; return; }
        if (prev != dev && cudaSetDevice(dev) != cudaSuccess) ok = false;
    }
    ~DeviceGuard()
    {
        int now = -1;
        if (prev >= 0 && cudaGetDevice(&now) == cudaSuccess && now != prev) cudaSetDevice(prev);
    }
};

void *dev_alloc(lbm13_t h, size_t bytes)
{
    bytes = (bytes + 255) & ~size_t(255);
    void *p = nullptr;
    if (h->has_alloc) {
        p = h->alloc.alloc(bytes, h->alloc.ctx);
    } else if (cudaMalloc(&p, bytes) != cudaSuccess) {
        cudaGetLastError();
        p = nullptr;
    }
    if (p) h->bytes_held += bytes;
    return p;
}

void dev_free(lbm13_t h, void *p, size_t bytes)
{
    if (!p) return;
    if (h->has_alloc) h->alloc.free(p, h->alloc.ctx);
    else cudaFree(p);
    bytes = (bytes + 255) & ~size_t(255);
    h->bytes_held -= bytes < h->bytes_held ? bytes : h->bytes_held;
}

bool finite_all(std::initializer_list<double> v)
{
    for (double x : v)
        if (!std::isfinite(x)) return false;
    return true;
}

// Sec. 2: Eqs. (d2q13-diffusion), (d2q13-sigma-qx), (d2q13-henon), and the shear
// relaxation time sigma_XX = 104 nu / A of the basis.  Fills out[] and returns a
// status: EINVAL for a rate outside (0, 2) or a non-positive viscosity, Prandtl
// number or A; EUNSTABLE when sigma_q <= 0.
// The rest-state scan of lbm13_create: wave vectors on a 9 x 9 grid of
// [-pi, pi]^2 (the edges, the origin and the diagonals included), and the
// round-off margin on |z| - 1.
constexpr int kCreateScanN = 9;
constexpr double kCreateScanTol = 1e-9;

int derive(const lbm13_params &p, double *out)
{
    for (int i = 0; i < LBM13_DERIVED_COUNT; ++i) out[i] = 0.0;
    const double E0 = p.E0, c1 = p.c1, k2 = p.k2, ceE = p.c_epsE;
    const double A = 13.0 * c1 + 95.0 + 2.0 * E0;
    const double B = 114404.0 + 51051.0 * c1 - 11492.0 * ceE + 7854.0 * E0;
    const double h1 = 17.0 / 26.0 - c1 / 2.0 - E0 / 13.0;
    const double k1 = 2.0 / 13.0;
    const double h2 = -(19.5 + 6.5 * c1 + E0) * k2 -
                      7.0 / 624.0 * A * (874481.0 + 459459.0 * c1 - 103428.0 * ceE + 70686.0 * E0) / B;
    const double sXX_sigma = 104.0 * p.nu / A;
    const double sq_sigma = -654.5 * sXX_sigma * A / B;
    const double cer = 140.0 + 28.0 * ceE + A * B / (22984.0 * p.Pr);
    const double c2 = -65.0 / 24.0 - 21.0 / 8.0 * (c1 + h1 + k1 * E0) - k2 * E0 - h2;
    const double sXX = 1.0 / (sXX_sigma + 0.5), sq = 1.0 / (sq_sigma + 0.5);
    out[0] = A; out[1] = B; out[2] = h1; out[3] = k1; out[4] = h2; out[5] = c2; out[6] = cer;
    out[7] = sXX_sigma; out[8] = sq_sigma;
    double s[Q] = {0, 0, p.s_eps, p.s_vpi, 0, 0, sq, sq, p.s_r, p.s_r, sXX, sXX, p.s_XXe};
    for (int k = 0; k < Q; ++k) out[9 + k] = s[k];
    // rest populations w = M^-1 (1, E0, eps0, varpi0, 0, ..., 0)
    Mom<double> d{};
    d.rho = 1.0 / kD[0];
    d.E = E0 / kD[1];
    d.eps = (cer + ceE * E0) / kD[2];
    d.vpi = (p.c_vpi_rho + p.c_vpi_E * E0) / kD[3];
    double w[Q] = {};
    inverse_add<true>(d, w);
    for (int j = 0; j < Q; ++j) out[22 + j] = w[j];
    out[35] = (E0 + 28.0) / 26.0;
    out[36] = A / 52.0;
    out[37] = p.nu / p.Pr;
    if (!finite_all({E0, c1, k2, ceE, p.c_vpi_rho, p.c_vpi_E, p.Pr, p.nu, p.s_eps, p.s_vpi, p.s_r, p.s_XXe}))
        return LBM13_EINVAL;
    if (!(A > 0.0) || !(p.nu > 0.0) || !(p.Pr > 0.0) || B == 0.0) return LBM13_EINVAL;
    if (!(sq_sigma > 0.0)) return LBM13_EUNSTABLE;
    const int nc[9] = {2, 3, 6, 7, 8, 9, 10, 11, 12};
    for (int i : nc)
        if (!(s[i] > 0.0 && s[i] < 2.0)) return LBM13_EINVAL;
    return LBM13_OK;
}

template <typename C>
void fill_coef(lbm13_t h, Coef<C> &k)
{
    collision_coef(h->p, h->derived, h->b, k);
}

template <typename C>
void fill_walls(lbm13_t h, WallArgs<C> *w)
{
    wall_coef(h->p, h->derived, h->b, h->kd, w);
}

template <typename T>
ReadArgs<T> read_args(lbm13_t h)
{
    ReadArgs<T> a;
    a.f = static_cast<const T *>(h->buf[h->cur]);
    a.nx = h->nx;
    a.ny = h->ny;
    a.pitch = h->pitch;
    a.plane = h->plane;
    a.rest.E0 = h->p.E0;
    a.rest.eps0 = h->derived[6] + h->p.c_epsE * h->p.E0;
    a.rest.vpi0 = h->p.c_vpi_rho + h->p.c_vpi_E * h->p.E0;
    a.gx = h->b.gx;
    a.gy = h->b.gy;
    a.rho_ref = h->b.rho_ref;
    a.heat = h->b.heat;
    return a;
}

// The same for rows y0 .. y1 - 1 only (a band of a banded read-out).
template <typename T>
ReadArgs<T> read_args_rows(lbm13_t h, int y0, int y1)
{
    ReadArgs<T> a = read_args<T>(h);
    a.f += (long long)y0 * h->pitch;
    a.ny = y1 - y0;
    return a;
}

// Host transfers of a lattice of kIoBandNodes nodes or more go in kIoBands row
// bands, the copies on the lattice's I/O stream overlapping the kernels of the
// neighbouring bands on its stream; smaller ones in one piece on its stream.
constexpr long long kIoBandNodes = 1LL << 22;
constexpr int kIoBands = 8;

// Band count for a transfer (*nb), and for banded ones the I/O stream and
// events (made on first use), the I/O stream ordered after the work already
// on the lattice's stream.
int io_prepare(lbm13_t h, int *nb)
{
    *nb = 1;
    if ((long long)h->nx * h->ny < kIoBandNodes || h->ny < kIoBands) return LBM13_OK;
    cudaError_t e = cudaSuccess;
    if (!h->io_stream) e = cudaStreamCreateWithFlags(&h->io_stream, cudaStreamNonBlocking);
    for (cudaEvent_t &ev : h->io_ev)
        if (e == cudaSuccess && !ev) e = cudaEventCreateWithFlags(&ev, cudaEventDisableTiming);
    if (e == cudaSuccess) e = cudaEventRecord(h->io_ev[2 * kIoBands], h->stream);
    if (e == cudaSuccess) e = cudaStreamWaitEvent(h->io_stream, h->io_ev[2 * kIoBands], 0);
    if (e != cudaSuccess) return cuda_fail(h, e, "I/O stream set-up");
    *nb = kIoBands;
    return LBM13_OK;
}

// Wait for a transfer's copies and kernels on both streams; the first error.
cudaError_t io_finish(lbm13_t h, int nb)
{
    cudaError_t a = nb > 1 ? cudaStreamSynchronize(h->io_stream) : cudaSuccess;
    cudaError_t b = cudaStreamSynchronize(h->stream);
    return a != cudaSuccess ? a : b;
}

template <typename T, typename C>
StepArgs<T, C> step_args(lbm13_t h, int cur, const Coef<C> &k, const WallArgs<C> *w)
{
    StepArgs<T, C> a{};
    a.fin = static_cast<const T *>(h->buf[cur]);
    a.fout = static_cast<T *>(h->buf[cur ^ 1]);
    a.nx = h->nx;
    a.ny = h->ny;
    a.per_x = h->b.west.kind == PERIODIC;
    a.per_y = h->b.south.kind == PERIODIC;
    a.pitch = h->pitch;
    a.plane = h->plane;
    a.k = k;
#ifdef LBM13_DEBUG
    a.bad = h->bad;
#endif
    for (int s = 0; s < 4; ++s) a.wall[s] = w[s];
    return a;
}

constexpr long long kGraphSteps = 32;  // even: a graph launch leaves the buffer parity unchanged

// Captures kGraphSteps step launches starting from buffer `cur` into a graph.
template <typename T, typename C>
cudaError_t build_graph(lbm13_t h, int cur, const Coef<C> &k, const WallArgs<C> *w)
{
    cudaError_t e;
    if (!h->cap_stream && (e = cudaStreamCreateWithFlags(&h->cap_stream, cudaStreamNonBlocking)) != cudaSuccess)
        return e;
    if ((e = cudaStreamBeginCapture(h->cap_stream, cudaStreamCaptureModeThreadLocal)) != cudaSuccess) return e;
    cudaError_t le = cudaSuccess;
    for (long long i = 0; i < kGraphSteps && le == cudaSuccess; ++i)
        le = launch_step<T, C>(step_args<T, C>(h, cur ^ int(i & 1), k, w), h->force, h->cap_stream);
    cudaGraph_t g = nullptr;
    e = cudaStreamEndCapture(h->cap_stream, &g);
    if (le != cudaSuccess) e = le;
    if (e == cudaSuccess) e = cudaGraphInstantiate(&h->gexec[cur], g, 0);
    if (g) cudaGraphDestroy(g);
    return e;
}

constexpr long long kPersistentChunk = 1024;  // steps per persistent launch (bounds a launch's duration)
constexpr unsigned long long kBarrierTimeoutNs = 1000000000ull;

GridSync grid_sync(lbm13_t h)
{
    unsigned *w = static_cast<unsigned *>(h->sync_mem);
    return GridSync{w, w + 32, w + 64, kBarrierTimeoutNs};
}

// The step launches' error word and grid-barrier words (made on first use).
bool ensure_sync_mem(lbm13_t h)
{
    if (h->sync_mem) return true;
    h->sync_mem = dev_alloc(h, kSyncBytes);
    if (!h->sync_mem) return false;
    return cudaMemsetAsync(h->sync_mem, 0, kSyncBytes, h->stream) == cudaSuccess;
}

template <typename T, typename C>
bool use_persistent(lbm13_t h, long long n)
{
    if (h->persistent != LBM13_PERSISTENT_ON || n < 2) return false;
    if (h->multi_grid < 0) h->multi_grid = multi_grid<T, C>(h->nx, h->ny, h->force);
    if (h->multi_grid <= 0) return false;
    return ensure_sync_mem(h);
}

// Reports (and clears) a grid-barrier timeout of an earlier persistent launch;
// the caller has synchronised the stream.
int check_barrier_error(lbm13_t h)
{
    if (!h->sync_mem) return LBM13_OK;
    unsigned err = 0;
    CK(h, cudaMemcpy(&err, static_cast<unsigned *>(h->sync_mem) + 64, sizeof(unsigned), cudaMemcpyDeviceToHost));
    if (err == 0) return LBM13_OK;
    CK(h, cudaMemset(h->sync_mem, 0, kSyncBytes));
    return fail(h, LBM13_ETIMEOUT,
                "a bounded wait of a step launch (a persistent launch's grid barrier or a paired step's tensor copy) "
                "timed out; the state is incomplete");
}

bool encode_pair_map(lbm13_t h, const void *buf, CUtensorMap *m);

// Whether lbm13_step pairs its steps: FP32, periodic in x and y, not in
// persistent mode, the tensor maps of both buffers made (once), and in AUTO
// mode a lattice of kPairMinNodes nodes or more (below that the persistent
// grid has too few tiles per block to hide each tile's copy: 256^2 to 768^2
// step faster singly; 1024^2 up 15%, 2048^2 up 25%, 8192^2 up 38%).
constexpr long long kPairMinNodes = 1LL << 20;

bool use_pairs(lbm13_t h)
{
    if (h->pair_mode == LBM13_PAIR_OFF || h->precision == LBM13_FP64 || h->persistent == LBM13_PERSISTENT_ON ||
        h->b.west.kind != PERIODIC || h->b.south.kind != PERIODIC)
        return false;
    if (h->pair_mode == LBM13_PAIR_AUTO && (long long)h->nx * h->ny < kPairMinNodes) return false;
    if (h->pair_ok < 0)
        h->pair_ok = encode_pair_map(h, h->buf[0], &h->pair_map[0]) && encode_pair_map(h, h->buf[1], &h->pair_map[1]);
    return h->pair_ok == 1;
}

unsigned *step_err(lbm13_t h) { return static_cast<unsigned *>(h->sync_mem) + 64; }

// Captures kGraphSteps / 2 paired launches starting from buffer `cur`.
cudaError_t build_pair_graph(lbm13_t h, int cur)
{
    cudaError_t e;
    if (!h->cap_stream && (e = cudaStreamCreateWithFlags(&h->cap_stream, cudaStreamNonBlocking)) != cudaSuccess)
        return e;
    if ((e = cudaStreamBeginCapture(h->cap_stream, cudaStreamCaptureModeThreadLocal)) != cudaSuccess) return e;
    cudaError_t le = cudaSuccess;
    for (long long i = 0; i < kGraphSteps / 2 && le == cudaSuccess; ++i) {
        const int b = cur ^ int(i & 1);
        le = launch_pair_step(step_args<float, float>(h, b, h->kf, h->wf), h->pair_map[b], h->force, step_err(h),
                              h->cap_stream);
    }
    cudaGraph_t g = nullptr;
    e = cudaStreamEndCapture(h->cap_stream, &g);
    if (le != cudaSuccess) e = le;
    if (e == cudaSuccess) e = cudaGraphInstantiate(&h->gexec2[cur], g, 0);
    if (g) cudaGraphDestroy(g);
    return e;
}

// n steps as paired launches (two steps each, the state's buffer flips at
// every launch), replayed from graphs of kGraphSteps steps, and a single step
// for an odd remainder.
int do_pair_steps(lbm13_t h, long long n)
{
    if (!ensure_sync_mem(h)) return fail(h, LBM13_ENOMEM, "allocator returned NULL for the step error word");
    if (n >= kGraphSteps) {
        if (!h->gexec2[h->cur]) {
            cudaError_t e = build_pair_graph(h, h->cur);
            if (e != cudaSuccess) return cuda_fail(h, e, "paired-step graph capture");
        }
        for (; n >= kGraphSteps; n -= kGraphSteps) {
            cudaError_t e = cudaGraphLaunch(h->gexec2[h->cur], h->stream);
            if (e != cudaSuccess) return cuda_fail(h, e, "cudaGraphLaunch (paired steps)");
            h->t += kGraphSteps;  // an even number of flips
        }
    }
    for (; n >= 2; n -= 2) {
        cudaError_t e = launch_pair_step(step_args<float, float>(h, h->cur, h->kf, h->wf), h->pair_map[h->cur],
                                         h->force, step_err(h), h->stream);
        if (e != cudaSuccess) return cuda_fail(h, e, "paired step launch");
        h->cur ^= 1;
        h->t += 2;
    }
    if (n == 1) {
        cudaError_t e = launch_step<float, float>(step_args<float, float>(h, h->cur, h->kf, h->wf), h->force, h->stream);
        if (e != cudaSuccess) return cuda_fail(h, e, "step kernel launch");
        h->cur ^= 1;
        h->t += 1;
    }
    return LBM13_OK;
}

template <typename T, typename C>
int do_steps(lbm13_t h, long long n, const Coef<C> &k, const WallArgs<C> *w)
{
    if (sizeof(T) == 4 && n >= 2 && use_pairs(h)) return do_pair_steps(h, n);
    if (use_persistent<T, C>(h, n)) {
        const GridSync g = grid_sync(h);
        while (n > 0) {
            const int m = int(n < kPersistentChunk ? n : kPersistentChunk);
            cudaError_t e = launch_multi<T, C>(step_args<T, C>(h, h->cur, k, w), step_args<T, C>(h, h->cur ^ 1, k, w),
                                               h->force, m, h->multi_grid, g, h->stream);
            if (e != cudaSuccess) return cuda_fail(h, e, "persistent step launch");
            h->cur ^= m & 1;
            h->t += m;
            n -= m;
        }
        return LBM13_OK;
    }
    if (n >= kGraphSteps) {
        if (!h->gexec[h->cur]) {
            cudaError_t e = build_graph<T, C>(h, h->cur, k, w);
            if (e != cudaSuccess) return cuda_fail(h, e, "step graph capture");
        }
        for (; n >= kGraphSteps; n -= kGraphSteps) {
            cudaError_t e = cudaGraphLaunch(h->gexec[h->cur], h->stream);
            if (e != cudaSuccess) return cuda_fail(h, e, "cudaGraphLaunch (steps)");
            h->t += kGraphSteps;
        }
    }
    for (long long i = 0; i < n; ++i) {
        cudaError_t e = launch_step<T, C>(step_args<T, C>(h, h->cur, k, w), h->force, h->stream);
        if (e != cudaSuccess) return cuda_fail(h, e, "step kernel launch");
        h->cur ^= 1;
        h->t += 1;
    }
    return LBM13_OK;
}

int check_wall(const lbm13_wall &w)
{
    return (w.kind == PERIODIC || w.kind == WALL_BB || w.kind == WALL_MIXED || w.kind == HALO) &&
           std::isfinite(w.u_t) && std::isfinite(w.T);
}

unsigned popcount18(unsigned m)
{
    unsigned c = 0;
    for (int b = 0; b < 18; ++b) c += (m >> b) & 1u;
    return c;
}

ReduceConf reduce_conf(lbm13_t h)
{
    ReduceConf c{};
    c.have_snap = h->have_snap;
    c.K = h->t - h->snap_t;
    c.step = h->t;
    const bool walls_T = h->b.west.kind == WALL_MIXED && h->b.east.kind == WALL_MIXED;
    c.nusselt = walls_T && h->b.west.T != h->b.east.T;
    c.dT = h->b.west.T - h->b.east.T;
    c.Tref = 0.5 * (h->b.west.T + h->b.east.T);
    c.kappa = h->p.nu / h->p.Pr;
    c.asym_walls = walls_T;
    c.Tasym = c.Tref;
    return c;
}

// The four reduction launches of one lattice, results to out_dev[16].
cudaError_t launch_residual(lbm13_t h, double *out_dev, cudaStream_t s)
{
    const ReduceConf c = reduce_conf(h);
    return h->precision == LBM13_FP64 ? launch_reduce<double>(read_args<double>(h), h->rb, c, out_dev, s)
                                      : launch_reduce<float>(read_args<float>(h), h->rb, c, out_dev, s);
}

int ensure_reduce(lbm13_t h)
{
    if (h->red_mem) return LBM13_OK;
    const long long n = (long long)h->nx * h->ny;
    const int nb = reduce_blocks(h->nx, h->ny);
    const size_t doubles = size_t(6 * n) + size_t(nb) * kPartials + 16 + 16;
    h->red_mem = dev_alloc(h, doubles * sizeof(double));
    if (!h->red_mem) return fail(h, LBM13_ENOMEM, "allocator returned NULL for the reduction buffers");
    double *base = static_cast<double *>(h->red_mem);
    h->rb.fields = base;
    h->rb.snap = base + 3 * n;
    h->rb.partials = base + 6 * n;
    h->rb.stats = h->rb.partials + size_t(nb) * kPartials;
    h->rb.nblocks = nb;
    h->out_dev = h->rb.stats + 16;
    return LBM13_OK;
}

} // namespace

extern "C" {

const char *lbm13_version(void) { return kVersion; }

const char *lbm13_status_string(int status)
{
    switch (status) {
    case LBM13_OK: return "ok";
    case LBM13_EINVAL: return "invalid argument";
    case LBM13_ENOMEM: return "out of device memory";
    case LBM13_EUNSTABLE: return "unstable parameter set";
    case LBM13_EDIVERGED: return "state diverged (non-finite populations)";
    case LBM13_ETIMEOUT: return "device-side wait timed out";
    case LBM13_ECUDA: return "CUDA error";
    default: return "unknown status";
    }
}

int lbm13_derive(const lbm13_params *params, double *out)
{
    if (!params || !out) return fail(nullptr, LBM13_EINVAL, "NULL argument");
    return derive(*params, out);
}

int lbm13_linear_growth(const lbm13_params *params, double ux, double uy, int n, double *growth)
{
    if (!params || !growth || n < 1 || n > 129) return fail(nullptr, LBM13_EINVAL, "NULL argument or n outside 1..129");
    double D[LBM13_DERIVED_COUNT];
    const int st = derive(*params, D);
    if (st != LBM13_OK) return fail(nullptr, st, "parameter set rejected by lbm13_derive");
    if (linear_growth(*params, D, ux, uy, n, growth) != LBM13_OK)
        return fail(nullptr, LBM13_EINVAL, "eigenvalue iteration did not converge");
    return LBM13_OK;
}

int lbm13_linear_growth_batch(const lbm13_params *params, const double *ux, const double *uy, int count, int n,
                              double *growth, void *stream)
{
    Range range_("lbm13_linear_growth_batch");
    if (!params || !ux || !uy || !growth || count < 1 || n < 1 || n > 129)
        return fail(nullptr, LBM13_EINVAL, "NULL argument, count < 1 or n outside 1..129");
    std::vector<double> D(size_t(count) * LBM13_DERIVED_COUNT);
    for (int c = 0; c < count; ++c) {
        if (!std::isfinite(ux[c]) || !std::isfinite(uy[c]))
            return fail(nullptr, LBM13_EINVAL, "non-finite background velocity");
        const int st = derive(params[c], D.data() + size_t(c) * LBM13_DERIVED_COUNT);
        if (st != LBM13_OK) return fail(nullptr, st, "a parameter set was rejected by lbm13_derive");
    }
    const int rc = linear_growth_batch(params, D.data(), ux, uy, count, n, growth, static_cast<cudaStream_t>(stream));
    if (rc == LBM13_EINVAL) return fail(nullptr, rc, "eigenvalue iteration did not converge");
    if (rc != LBM13_OK) return fail(nullptr, rc, "CUDA error in the batched stability scan");
    return LBM13_OK;
}

const char *lbm13_last_error(lbm13_t h) { return h ? h->err.c_str() : g_err.c_str(); }

int lbm13_debug_violations(lbm13_t h, unsigned long long *count)
{
    if (!h || !count) return fail(h, LBM13_EINVAL, "NULL argument");
#ifdef LBM13_DEBUG
    DeviceGuard g(h->device);
    cudaError_t e = cudaMemcpyAsync(count, h->bad, sizeof(unsigned long long), cudaMemcpyDeviceToHost, h->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(h->stream);
    if (e != cudaSuccess) return cuda_fail(h, e, "debug access counter");
    return LBM13_OK;
#else
    *count = 0;
    return fail(h, LBM13_EINVAL, "built without LBM13_DEBUG: population accesses are not checked");
#endif
}

int lbm13_create(int nx, int ny, const lbm13_params *params, const lbm13_boundary *boundary, int precision,
                 const lbm13_allocator *alloc, void *stream, lbm13_t *out)
{
    if (!out) return fail(nullptr, LBM13_EINVAL, "out is NULL");
    *out = nullptr;
    if (!params || !boundary) return fail(nullptr, LBM13_EINVAL, "params or boundary is NULL");
    if (precision != LBM13_FP64 && precision != LBM13_FP32_DEVIATION)
        return fail(nullptr, LBM13_EINVAL, "precision must be LBM13_FP64 or LBM13_FP32_DEVIATION");
    const lbm13_boundary &b = *boundary;
    if (!check_wall(b.west) || !check_wall(b.east) || !check_wall(b.south) || !check_wall(b.north) ||
        !finite_all({b.gx, b.gy, b.rho_ref, b.heat}))
        return fail(nullptr, LBM13_EINVAL, "bad wall kind or non-finite boundary data");
    if (b.wall_density != LBM13_WALL_DENSITY_EXTRAPOLATE && b.wall_density != LBM13_WALL_DENSITY_ZERO_FLUX)
        return fail(nullptr, LBM13_EINVAL, "wall_density must be LBM13_WALL_DENSITY_EXTRAPOLATE or _ZERO_FLUX");
    if ((b.west.kind == PERIODIC) != (b.east.kind == PERIODIC) || (b.south.kind == PERIODIC) != (b.north.kind == PERIODIC))
        return fail(nullptr, LBM13_EINVAL, "opposite sides must both be periodic or both be walls");
    if (b.west.kind == HALO || b.east.kind == HALO)
        return fail(nullptr, LBM13_EINVAL, "halo sides (y-slabs) are south or north only");
    const int halos = (b.south.kind == HALO) + (b.north.kind == HALO);
    const int min_x = b.west.kind == PERIODIC ? 2 : 4, min_y = b.south.kind == PERIODIC ? 2 : 4 + 2 * halos;
    if (nx < min_x || ny < min_y || nx > (1 << 20) || ny > 32768 || (long long)nx * ny > 0x7fffffffLL)
        return fail(nullptr, LBM13_EINVAL,
                    "lattice size out of range (>= 2, >= 4 along a walled axis plus 2 rows per halo side, nx <= 2^20, "
                    "ny <= 32768, nx*ny < 2^31)");
    if (alloc && (!alloc->alloc || !alloc->free)) return fail(nullptr, LBM13_EINVAL, "allocator without alloc/free");

    lbm13_t h = new lbm13_lattice();
    h->nx = nx;
    h->ny = ny;
    h->precision = precision;
    h->p = *params;
    h->b = b;
    if (alloc) { h->alloc = *alloc; h->has_alloc = true; }
    h->stream = static_cast<cudaStream_t>(stream);
    int st = derive(h->p, h->derived);
    if (st != LBM13_OK) {
        delete h;
        return fail(nullptr, st, st == LBM13_EUNSTABLE ? "sigma_q <= 0: no positive relaxation time for q"
                                                       : "parameter out of range (rates in (0,2), nu > 0, Pr > 0)");
    }
    // the linearised step must not amplify any Fourier mode at rest, nor in a
    // uniform flow at the largest wall speed along either axis
    const double uw = std::max({std::fabs(b.west.u_t), std::fabs(b.east.u_t), std::fabs(b.south.u_t),
                                std::fabs(b.north.u_t)});
    const double scan_u[3][2] = {{0.0, 0.0}, {uw, 0.0}, {0.0, uw}};
    for (int k = 0; k < (uw > 0.0 ? 3 : 1); ++k) {
        double growth = 0.0;
        if (linear_growth(h->p, h->derived, scan_u[k][0], scan_u[k][1], kCreateScanN, &growth) != LBM13_OK ||
            !(growth <= kCreateScanTol)) {
            delete h;
            char msg[200];
            std::snprintf(msg, sizeof msg,
                          "linearly unstable at u = (%.3g, %.3g): max |z| - 1 = %.3g over a %d x %d k-grid",
                          scan_u[k][0], scan_u[k][1], growth, kCreateScanN, kCreateScanN);
            return fail(nullptr, LBM13_EUNSTABLE, msg);
        }
    }
    if (cudaGetDevice(&h->device) != cudaSuccess) {
        cudaGetLastError();
        delete h;
        return fail(nullptr, LBM13_ECUDA, "no CUDA device");
    }
    fill_coef(h, h->kd);
    fill_coef(h, h->kf);
    fill_walls(h, h->wd);
    fill_walls(h, h->wf);
    h->force = h->b.gx != 0.0 || h->b.gy != 0.0 || h->b.heat != 0.0;
    h->elem = precision == LBM13_FP64 ? sizeof(double) : sizeof(float);
    h->pitch = ((long long)nx + 31) / 32 * 32;
    h->plane = (long long)ny * h->pitch;
    h->state_bytes = size_t(Q) * size_t(h->plane) * h->elem;
    for (int i = 0; i < 2; ++i) {
        h->buf[i] = dev_alloc(h, h->state_bytes);
        if (!h->buf[i]) {
            lbm13_destroy(h);
            return fail(nullptr, LBM13_ENOMEM, "allocator returned NULL for the population buffers");
        }
    }
#ifdef LBM13_DEBUG
    h->bad = static_cast<unsigned long long *>(dev_alloc(h, sizeof(unsigned long long)));
    if (!h->bad || cudaMemsetAsync(h->bad, 0, sizeof(unsigned long long), h->stream) != cudaSuccess) {
        lbm13_destroy(h);
        return fail(nullptr, LBM13_ENOMEM, "debug access counter");
    }
#endif
    // deviation 0 everywhere = the rest state rho = 1, u = 0, T = T0
    for (int i = 0; i < 2; ++i) {
        cudaError_t e = cudaMemsetAsync(h->buf[i], 0, h->state_bytes, h->stream);
        if (e != cudaSuccess) {
            lbm13_destroy(h);
            return cuda_fail(nullptr, e, "cudaMemsetAsync");
        }
    }
    *out = h;
    return LBM13_OK;
}

void lbm13_destroy(lbm13_t h)
{
    if (!h) return;
    DeviceGuard g(h->device);
    cudaStreamSynchronize(h->stream);
    for (int i = 0; i < 2; ++i) {
        if (h->gexec[i]) cudaGraphExecDestroy(h->gexec[i]);
        if (h->gexec2[i]) cudaGraphExecDestroy(h->gexec2[i]);
    }
    if (h->cap_stream) cudaStreamDestroy(h->cap_stream);
    if (h->io_stream) {
        cudaStreamSynchronize(h->io_stream);
        cudaStreamDestroy(h->io_stream);
    }
    for (cudaEvent_t ev : h->io_ev)
        if (ev) cudaEventDestroy(ev);
    for (int i = 0; i < 2; ++i) dev_free(h, h->buf[i], h->state_bytes);
    if (h->bad) dev_free(h, h->bad, sizeof(unsigned long long));
    if (h->red_mem) {
        const long long n = (long long)h->nx * h->ny;
        dev_free(h, h->red_mem, (size_t(6 * n) + size_t(h->rb.nblocks) * kPartials + 32) * sizeof(double));
    }
    if (h->proj_mem) dev_free(h, h->proj_mem, size_t(h->proj_blocks + 1) * kProj * sizeof(double));
    if (h->sync_mem) dev_free(h, h->sync_mem, kSyncBytes);
    delete h;
}

int lbm13_set_stream(lbm13_t h, void *stream)
{
    if (!h) return fail(nullptr, LBM13_EINVAL, "NULL handle");
    h->stream = static_cast<cudaStream_t>(stream);
    return LBM13_OK;
}

int lbm13_info(lbm13_t h, int64_t out[8])
{
    if (!h || !out) return fail(h, LBM13_EINVAL, "NULL argument");
    out[0] = h->nx;
    out[1] = h->ny;
    out[2] = h->pitch;
    out[3] = h->precision;
    out[4] = (int64_t)h->elem;
    out[5] = (int64_t)h->bytes_held;
    out[6] = h->t;
    out[7] = h->multi_grid > 0 ? h->multi_grid : 0;
    return LBM13_OK;
}

int lbm13_step_launches(lbm13_t h, int64_t n, int64_t *launches)
{
    if (!h || !launches || n < 0) return fail(h, LBM13_EINVAL, "NULL argument or negative step count");
    DeviceGuard g(h->device);
    if (n >= 2 && h->precision != LBM13_FP64 && use_pairs(h))
        *launches = n / 2 + (n & 1);
    else if (n >= 2 && (h->precision == LBM13_FP64 ? use_persistent<double, double>(h, n)
                                                     : use_persistent<float, float>(h, n)))
        *launches = (n + kPersistentChunk - 1) / kPersistentChunk;
    else
        *launches = n;
    return LBM13_OK;
}

int lbm13_set_pair_steps(lbm13_t h, int mode)
{
    if (!h) return fail(nullptr, LBM13_EINVAL, "NULL handle");
    if (mode != LBM13_PAIR_AUTO && mode != LBM13_PAIR_OFF && mode != LBM13_PAIR_ON)
        return fail(h, LBM13_EINVAL, "mode must be LBM13_PAIR_AUTO, LBM13_PAIR_OFF or LBM13_PAIR_ON");
    h->pair_mode = mode;
    return LBM13_OK;
}

int lbm13_pair_check(lbm13_t h, double timeout_s, int withhold, int *timed_out)
{
    if (!h || !timed_out || !(timeout_s >= 1e-3 && timeout_s <= 2.0))
        return fail(h, LBM13_EINVAL, "NULL argument or timeout_s outside [1e-3, 2]");
    DeviceGuard g(h->device);
    if (!use_pairs(h)) return fail(h, LBM13_EINVAL, "the lattice does not take paired steps");
    if (!ensure_sync_mem(h)) return fail(h, LBM13_ENOMEM, "allocator returned NULL for the step error word");
    CK(h, cudaStreamSynchronize(h->stream));
    int rc = check_barrier_error(h);
    if (rc != LBM13_OK) return rc;
    cudaError_t e = launch_pair_step(step_args<float, float>(h, h->cur, h->kf, h->wf), h->pair_map[h->cur], h->force,
                                     step_err(h), h->stream, withhold ? 0 : 1,
                                     (unsigned long long)(timeout_s * 1e9));
    if (e == cudaSuccess) e = cudaStreamSynchronize(h->stream);
    unsigned word = 0;
    if (e == cudaSuccess) e = cudaMemcpy(&word, step_err(h), sizeof word, cudaMemcpyDeviceToHost);
    if (e == cudaSuccess) e = cudaMemset(h->sync_mem, 0, kSyncBytes);
    if (e != cudaSuccess) return cuda_fail(h, e, "paired-step check");
    *timed_out = word != 0u;
    return LBM13_OK;
}

int lbm13_set_persistent(lbm13_t h, int mode)
{
    if (!h) return fail(nullptr, LBM13_EINVAL, "NULL handle");
    if (mode != LBM13_PERSISTENT_AUTO && mode != LBM13_PERSISTENT_OFF && mode != LBM13_PERSISTENT_ON)
        return fail(h, LBM13_EINVAL, "mode must be LBM13_PERSISTENT_AUTO, _OFF or _ON");
    h->persistent = mode;
    return LBM13_OK;
}

int lbm13_barrier_check(int blocks, int extra_blocks, double timeout_s, int *timed_out)
{
    if (!timed_out || blocks < 1 || blocks > 1024 || extra_blocks < 0 || extra_blocks > 1024 ||
        !(timeout_s >= 1e-3 && timeout_s <= 2.0))
        return fail(nullptr, LBM13_EINVAL, "blocks in 1..1024, extra_blocks in 0..1024, timeout_s in [1e-3, 2]");
    void *mem = nullptr;
    cudaError_t e = cudaMalloc(&mem, kSyncBytes);
    if (e != cudaSuccess) return cuda_fail(nullptr, e, "cudaMalloc (barrier words)");
    unsigned *w = static_cast<unsigned *>(mem);
    const GridSync g{w, w + 32, w + 64, (unsigned long long)(timeout_s * 1e9)};
    unsigned err = 0;
    e = cudaMemset(mem, 0, kSyncBytes);
    if (e == cudaSuccess) e = launch_barrier_check(blocks, unsigned(blocks + extra_blocks), 4, g, nullptr);
    if (e == cudaSuccess) e = cudaDeviceSynchronize();
    if (e == cudaSuccess) e = cudaMemcpy(&err, w + 64, sizeof(unsigned), cudaMemcpyDeviceToHost);
    cudaFree(mem);
    if (e != cudaSuccess) return cuda_fail(nullptr, e, "barrier check");
    *timed_out = err != 0u;
    return LBM13_OK;
}

int lbm13_set_state_device(lbm13_t h, const double *rho, const double *ux, const double *uy, const double *T)
{
    if (!h || !rho || !ux || !uy || !T) return fail(h, LBM13_EINVAL, "NULL argument");
    DeviceGuard g(h->device);
    cudaError_t e;
    if (h->precision == LBM13_FP64)
        e = launch_init<double>(static_cast<double *>(h->buf[h->cur]), h->nx, h->ny, h->pitch, h->plane, h->kd, rho,
                                ux, uy, T, h->stream);
    else
        e = launch_init<float>(static_cast<float *>(h->buf[h->cur]), h->nx, h->ny, h->pitch, h->plane, h->kd, rho,
                               ux, uy, T, h->stream);
    if (e != cudaSuccess) return cuda_fail(h, e, "init kernel launch");
    h->t = 0;
    h->have_snap = 0;
    return LBM13_OK;
}

int lbm13_set_state(lbm13_t h, const double *rho, const double *ux, const double *uy, const double *T)
{
    Range range_("lbm13_set_state");
    if (!h) return fail(nullptr, LBM13_EINVAL, "NULL handle");
    DeviceGuard g(h->device);
    const size_t n = size_t(h->nx) * h->ny, bytes = n * sizeof(double);
    double *stage = static_cast<double *>(dev_alloc(h, 4 * bytes));
    if (!stage) return fail(h, LBM13_ENOMEM, "allocator returned NULL for the state staging buffer");
    const double rest[4] = {1.0, 0.0, 0.0, (h->p.E0 + 28.0) / 26.0};
    const double *src[4] = {rho, ux, uy, T};
    std::vector<double> fill[4];  // absent fields: uniform, alive until the copies are done
    for (int q = 0; q < 4; ++q)
        if (!src[q]) {
            fill[q].assign(n, rest[q]);
            src[q] = fill[q].data();
        }
    int nb = 1;
    int rc = io_prepare(h, &nb);
    const int rows = (h->ny + nb - 1) / nb;
    for (int b = 0; b < nb && rc == LBM13_OK; ++b) {
        // band b: rows y0 .. y1 - 1 of the four fields, uploaded on the I/O
        // stream (the first band's copies wait for the work already on the
        // lattice's stream), then initialised on the lattice's stream
        const int y0 = b * rows, y1 = std::min(h->ny, y0 + rows);
        if (y0 >= y1) break;
        const size_t off = size_t(y0) * h->nx, cnt = size_t(y1 - y0) * h->nx;
        cudaStream_t cs = nb > 1 ? h->io_stream : h->stream;
        cudaError_t e = cudaSuccess;
        for (int q = 0; q < 4 && e == cudaSuccess; ++q)
            e = cudaMemcpyAsync(stage + q * n + off, src[q] + off, cnt * sizeof(double), cudaMemcpyHostToDevice, cs);
        if (e == cudaSuccess && nb > 1) e = cudaEventRecord(h->io_ev[b], cs);
        if (e == cudaSuccess && nb > 1) e = cudaStreamWaitEvent(h->stream, h->io_ev[b], 0);
        if (e != cudaSuccess) {
            rc = cuda_fail(h, e, "cudaMemcpyAsync (state upload)");
            break;
        }
        e = h->precision == LBM13_FP64
                ? launch_init<double>(static_cast<double *>(h->buf[h->cur]) + (long long)y0 * h->pitch, h->nx, y1 - y0,
                                      h->pitch, h->plane, h->kd, stage + off, stage + n + off, stage + 2 * n + off,
                                      stage + 3 * n + off, h->stream)
                : launch_init<float>(static_cast<float *>(h->buf[h->cur]) + (long long)y0 * h->pitch, h->nx, y1 - y0,
                                     h->pitch, h->plane, h->kd, stage + off, stage + n + off, stage + 2 * n + off,
                                     stage + 3 * n + off, h->stream);
        if (e != cudaSuccess) rc = cuda_fail(h, e, "init kernel launch");
    }
    if (rc == LBM13_OK) {
        h->t = 0;
        h->have_snap = 0;
    }
    cudaError_t e = io_finish(h, nb);
    if (rc == LBM13_OK && e != cudaSuccess) rc = cuda_fail(h, e, "cudaStreamSynchronize (set_state)");
    dev_free(h, stage, 4 * bytes);
    return rc;
}

int lbm13_set_raw_state(lbm13_t h, const double *f, int64_t step)
{
    if (!h || !f) return fail(h, LBM13_EINVAL, "NULL argument");
    DeviceGuard g(h->device);
    const double *w = h->derived + 22;
    const size_t n = size_t(h->nx) * h->ny;
    std::vector<unsigned char> host(h->state_bytes, 0);
    for (int j = 0; j < Q; ++j)
        for (int y = 0; y < h->ny; ++y)
            for (int x = 0; x < h->nx; ++x) {
                const double v = f[size_t(j) * n + size_t(y) * h->nx + x] - w[j];
                const size_t at = size_t(j) * h->plane + size_t(y) * h->pitch + x;
                if (h->precision == LBM13_FP64) reinterpret_cast<double *>(host.data())[at] = v;
                else reinterpret_cast<float *>(host.data())[at] = float(v);
            }
    CK(h, cudaStreamSynchronize(h->stream));
    CK(h, cudaMemcpy(h->buf[h->cur], host.data(), h->state_bytes, cudaMemcpyHostToDevice));
    h->t = step;
    h->have_snap = 0;
    return LBM13_OK;
}

int lbm13_get_raw_state(lbm13_t h, double *f, int64_t *step)
{
    if (!h || !f) return fail(h, LBM13_EINVAL, "NULL argument");
    DeviceGuard g(h->device);
    const double *w = h->derived + 22;
    const size_t n = size_t(h->nx) * h->ny;
    std::vector<unsigned char> host(h->state_bytes);
    SYNC_CHECK(h);
    CK(h, cudaMemcpy(host.data(), h->buf[h->cur], h->state_bytes, cudaMemcpyDeviceToHost));
    for (int j = 0; j < Q; ++j)
        for (int y = 0; y < h->ny; ++y)
            for (int x = 0; x < h->nx; ++x) {
                const size_t at = size_t(j) * h->plane + size_t(y) * h->pitch + x;
                const double v = h->precision == LBM13_FP64 ? reinterpret_cast<const double *>(host.data())[at]
                                                            : double(reinterpret_cast<const float *>(host.data())[at]);
                f[size_t(j) * n + size_t(y) * h->nx + x] = v + w[j];
            }
    if (step) *step = h->t;
    return LBM13_OK;
}

int lbm13_checkpoint_bytes(lbm13_t h, size_t *bytes)
{
    if (!h || !bytes) return fail(h, LBM13_EINVAL, "NULL argument");
    *bytes = 64 + h->state_bytes;
    return LBM13_OK;
}

static const char kMagic[8] = {'L', 'B', 'M', '1', '3', 'C', 'K', '1'};

int lbm13_save(lbm13_t h, void *host, size_t bytes)
{
    if (!h || !host) return fail(h, LBM13_EINVAL, "NULL argument");
    if (bytes < 64 + h->state_bytes) return fail(h, LBM13_EINVAL, "checkpoint buffer too small");
    DeviceGuard g(h->device);
    unsigned char *p = static_cast<unsigned char *>(host);
    int64_t hdr[8] = {0, h->nx, h->ny, h->precision, h->pitch, h->t, 0, 0};
    std::memcpy(hdr, kMagic, 8);
    std::memcpy(p, hdr, 64);
    SYNC_CHECK(h);
    CK(h, cudaMemcpy(p + 64, h->buf[h->cur], h->state_bytes, cudaMemcpyDeviceToHost));
    return LBM13_OK;
}

int lbm13_restore(lbm13_t h, const void *host, size_t bytes)
{
    if (!h || !host) return fail(h, LBM13_EINVAL, "NULL argument");
    if (bytes < 64 + h->state_bytes) return fail(h, LBM13_EINVAL, "checkpoint image too small");
    const unsigned char *p = static_cast<const unsigned char *>(host);
    int64_t hdr[8];
    std::memcpy(hdr, p, 64);
    if (std::memcmp(hdr, kMagic, 8) != 0 || hdr[1] != h->nx || hdr[2] != h->ny || hdr[3] != h->precision ||
        hdr[4] != h->pitch)
        return fail(h, LBM13_EINVAL, "checkpoint image does not match this lattice");
    DeviceGuard g(h->device);
    CK(h, cudaStreamSynchronize(h->stream));
    CK(h, cudaMemcpy(h->buf[h->cur], p + 64, h->state_bytes, cudaMemcpyHostToDevice));
    h->t = hdr[5];
    h->have_snap = 0;
    return LBM13_OK;
}

int lbm13_step(lbm13_t h, int64_t n)
{
    Range range_("lbm13_step");
    if (!h || n < 0) return fail(h, LBM13_EINVAL, "NULL handle or negative step count");
    if (n == 0) return LBM13_OK;
    DeviceGuard g(h->device);
    if (h->precision == LBM13_FP64) return do_steps<double, double>(h, n, h->kd, h->wd);
    return do_steps<float, float>(h, n, h->kf, h->wf);
}

int lbm13_moments_device(lbm13_t h, double *out, unsigned mask)
{
    if (!h || !out) return fail(h, LBM13_EINVAL, "NULL argument");
    if (mask == 0 || (mask >> 18) != 0) return fail(h, LBM13_EINVAL, "mask must select bits 0..17");
    DeviceGuard g(h->device);
    cudaError_t e = h->precision == LBM13_FP64 ? launch_moments<double>(read_args<double>(h), out, mask, h->stream)
                                               : launch_moments<float>(read_args<float>(h), out, mask, h->stream);
    if (e != cudaSuccess) return cuda_fail(h, e, "moments kernel launch");
    return LBM13_OK;
}

int lbm13_moments(lbm13_t h, double *out, unsigned mask)
{
    Range range_("lbm13_moments");
    if (!h || !out) return fail(h, LBM13_EINVAL, "NULL argument");
    if (mask == 0 || (mask >> 18) != 0) return fail(h, LBM13_EINVAL, "mask must select bits 0..17");
    DeviceGuard g(h->device);
    const int nf = popcount18(mask);
    const size_t n = size_t(h->nx) * h->ny, bytes = size_t(nf) * n * sizeof(double);
    double *stage = static_cast<double *>(dev_alloc(h, bytes));
    if (!stage) return fail(h, LBM13_ENOMEM, "allocator returned NULL for the moments staging buffer");
    int nb = 1;
    int rc = io_prepare(h, &nb);
    const int rows = (h->ny + nb - 1) / nb;
    for (int b = 0; b < nb && rc == LBM13_OK; ++b) {
        // band b: its fields computed on the lattice's stream into a block of
        // the staging buffer laid out [field][rows][nx], then downloaded on
        // the I/O stream while the next band is computed
        const int y0 = b * rows, y1 = std::min(h->ny, y0 + rows);
        if (y0 >= y1) break;
        const size_t off = size_t(y0) * h->nx, cnt = size_t(y1 - y0) * h->nx;
        double *blk = stage + off * nf;
        cudaError_t e = h->precision == LBM13_FP64
                            ? launch_moments<double>(read_args_rows<double>(h, y0, y1), blk, mask, h->stream)
                            : launch_moments<float>(read_args_rows<float>(h, y0, y1), blk, mask, h->stream);
        if (e != cudaSuccess) {
            rc = cuda_fail(h, e, "moments kernel launch");
            break;
        }
        cudaStream_t cs = nb > 1 ? h->io_stream : h->stream;
        if (nb > 1) e = cudaEventRecord(h->io_ev[nb + b], h->stream);
        if (e == cudaSuccess && nb > 1) e = cudaStreamWaitEvent(cs, h->io_ev[nb + b], 0);
        for (int k = 0; k < nf && e == cudaSuccess; ++k)
            e = cudaMemcpyAsync(out + k * n + off, blk + k * cnt, cnt * sizeof(double), cudaMemcpyDeviceToHost, cs);
        if (e != cudaSuccess) rc = cuda_fail(h, e, "moments download");
    }
    cudaError_t e = io_finish(h, nb);
    if (rc == LBM13_OK && e != cudaSuccess) rc = cuda_fail(h, e, "moments download");
    if (rc == LBM13_OK) rc = check_barrier_error(h);
    dev_free(h, stage, bytes);
    return rc;
}

int lbm13_residual(lbm13_t h, double *out)
{
    Range range_("lbm13_residual");
    if (!h || !out) return fail(h, LBM13_EINVAL, "NULL argument");
    DeviceGuard g(h->device);
    int rc = ensure_reduce(h);
    if (rc != LBM13_OK) return rc;
    cudaError_t e = launch_residual(h, h->out_dev, h->stream);
    if (e != cudaSuccess) return cuda_fail(h, e, "reduction kernel launch");
    CK(h, cudaMemcpyAsync(out, h->out_dev, 16 * sizeof(double), cudaMemcpyDeviceToHost, h->stream));
    SYNC_CHECK(h);
    h->have_snap = 1;
    h->snap_t = h->t;
    if (out[LBM13_R_NONFINITE] > 0.0) return fail(h, LBM13_EDIVERGED, "non-finite populations in the state");
    return LBM13_OK;
}

int lbm13_project(lbm13_t h, int kx, int ky, double *out)
{
    Range range_("lbm13_project");
    if (!h || !out) return fail(h, LBM13_EINVAL, "NULL argument");
    DeviceGuard g(h->device);
    if (!h->proj_mem) {
        const int nb = reduce_blocks(h->nx, h->ny);
        h->proj_mem = dev_alloc(h, size_t(nb + 1) * kProj * sizeof(double));
        if (!h->proj_mem) return fail(h, LBM13_ENOMEM, "allocator returned NULL for the projection buffers");
        h->proj_blocks = nb;
    }
    double *partials = static_cast<double *>(h->proj_mem);
    double *res = partials + size_t(h->proj_blocks) * kProj;
    cudaError_t e = h->precision == LBM13_FP64
                        ? launch_project<double>(read_args<double>(h), kx, ky, partials, h->proj_blocks, res, h->stream)
                        : launch_project<float>(read_args<float>(h), kx, ky, partials, h->proj_blocks, res, h->stream);
    if (e != cudaSuccess) return cuda_fail(h, e, "projection kernel launch");
    CK(h, cudaMemcpyAsync(out, res, kProj * sizeof(double), cudaMemcpyDeviceToHost, h->stream));
    SYNC_CHECK(h);
    return LBM13_OK;
}

int64_t lbm13_time(lbm13_t h) { return h ? h->t : -1; }

int lbm13_synchronize(lbm13_t h)
{
    if (!h) return fail(nullptr, LBM13_EINVAL, "NULL handle");
    DeviceGuard g(h->device);
    SYNC_CHECK(h);
    return LBM13_OK;
}

} // extern "C"

bool lbm13_state_view(const lbm13_lattice *h, lbm13::StateView *v)
{
    if (!h || !v) return false;
    v->f = h->buf[h->cur];
    v->nx = h->nx;
    v->ny = h->ny;
    v->precision = h->precision;
    v->device = h->device;
    v->pitch = h->pitch;
    v->plane = h->plane;
    v->E0 = h->p.E0;
    v->gx = h->b.gx;
    v->gy = h->b.gy;
    v->rho_ref = h->b.rho_ref;
    v->heat = h->b.heat;
    v->stream = h->stream;
    return true;
}

// ------------------------------------------------------------ y-slab halos

namespace {

int halo_check(lbm13_t h, int side, const void *buf)
{
    if (!h || !buf) return fail(h, LBM13_EINVAL, "NULL argument");
    if (side != LBM13_HALO_SOUTH && side != LBM13_HALO_NORTH) return fail(h, LBM13_EINVAL, "side must be south or north");
    const lbm13_wall &w = side == LBM13_HALO_SOUTH ? h->b.south : h->b.north;
    if (w.kind != HALO) return fail(h, LBM13_EINVAL, "that side of the lattice is not a halo side");
    return LBM13_OK;
}

int halo_move(lbm13_t h, int side, void *buf, bool pack)
{
    DeviceGuard g(h->device);
    const int s = side == LBM13_HALO_SOUTH ? SOUTH : NORTH;
    cudaError_t e = h->precision == LBM13_FP64
                        ? launch_halo<double>(static_cast<double *>(h->buf[h->cur]), h->nx, h->ny, h->pitch, h->plane,
                                              s, pack, static_cast<double *>(buf), h->stream)
                        : launch_halo<float>(static_cast<float *>(h->buf[h->cur]), h->nx, h->ny, h->pitch, h->plane, s,
                                             pack, static_cast<float *>(buf), h->stream);
    if (e != cudaSuccess) return fail(h, LBM13_ECUDA, std::string("halo launch: ") + cudaGetErrorString(e));
    return LBM13_OK;
}

} // namespace

extern "C" {

int lbm13_halo_bytes(lbm13_t h, size_t *bytes)
{
    if (!h || !bytes) return fail(h, LBM13_EINVAL, "NULL argument");
    *bytes = size_t(8) * size_t(h->nx) * h->elem;
    return LBM13_OK;
}

int lbm13_halo_pack(lbm13_t h, int side, void *out)
{
    Range range_("lbm13_halo_pack");
    const int rc = halo_check(h, side, out);
    return rc != LBM13_OK ? rc : halo_move(h, side, out, true);
}

int lbm13_halo_unpack(lbm13_t h, int side, const void *in)
{
    Range range_("lbm13_halo_unpack");
    const int rc = halo_check(h, side, in);
    return rc != LBM13_OK ? rc : halo_move(h, side, const_cast<void *>(in), false);
}

} // extern "C"

// ------------------------------------------------------------------ plans
//
// A plan steps many lattices with one batched launch per time step.  The
// device table holds every lattice's arguments for both buffer parities; the
// work list holds (lattice, tile) pairs in the order chosen by the tuner.

struct lbm13_plan {
    std::vector<lbm13_t> lats;
    int precision = 0, device = 0;
    cudaStream_t stream = nullptr;
    lbm13_allocator alloc{};
    bool has_alloc = false;
    void *desc = nullptr;
    size_t desc_bytes = 0;
    void *work = nullptr;
    size_t work_bytes = 0;
    int ntiles = 0;
    double *res_dev = nullptr;  // [res_cap][16] results of lbm13_plan_residual
    size_t res_cap = 0;
    size_t cap = 0;             // lattices the device table (and maps) can hold
    cudaEvent_t order_ev = nullptr;  // orders a lattice's own stream against the plan's
    long long nodes = 0;
    std::vector<int> cur0;
    int parity = 0;  // parity of the next launch relative to cur0
    int R = 2, BY = 4, ctas = 8, order = 0, groups = 1, grid = 0, sms = 0, tried = 0;
    // FP32: the lattices' tensor maps for the staged tiles (R = 4, BY = 4, one
    // block per tile) and the word their bounded waits set when one runs out
    void *maps = nullptr;
    size_t maps_bytes = 0;
    // per lattice, the ring-staged maps made: bit 0 the 64-column strips',
    // bit 1 the 32-column strips' (the edge work items follow them)
    std::vector<unsigned char> ring_ok;
    unsigned *tma_err = nullptr;
    cudaStream_t cap_stream = nullptr;
    cudaGraphExec_t gexec[2] = {nullptr, nullptr};
    std::string err;
};

namespace {

int pfail(lbm13_plan_t p, int code, const std::string &msg)
{
    if (p) p->err = msg;
    g_err = msg;
    return code;
}

void *plan_alloc(lbm13_plan_t p, size_t bytes)
{
    bytes = (bytes + 255) & ~size_t(255);
    void *ptr = nullptr;
    if (p->has_alloc) ptr = p->alloc.alloc(bytes, p->alloc.ctx);
    else if (cudaMalloc(&ptr, bytes) != cudaSuccess) { cudaGetLastError(); ptr = nullptr; }
    return ptr;
}

void plan_free(lbm13_plan_t p, void *ptr)
{
    if (!ptr) return;
    if (p->has_alloc) p->alloc.free(ptr, p->alloc.ctx);
    else cudaFree(ptr);
}

template <typename C> const Coef<C> &coef_of(lbm13_t h);
template <> const Coef<double> &coef_of<double>(lbm13_t h) { return h->kd; }
template <> const Coef<float> &coef_of<float>(lbm13_t h) { return h->kf; }
template <typename C> const WallArgs<C> *walls_of(lbm13_t h);
template <> const WallArgs<double> *walls_of<double>(lbm13_t h) { return h->wd; }
template <> const WallArgs<float> *walls_of<float>(lbm13_t h) { return h->wf; }

void plan_drop_graphs(lbm13_plan_t p)
{
    for (int i = 0; i < 2; ++i)
        if (p->gexec[i]) { cudaGraphExecDestroy(p->gexec[i]); p->gexec[i] = nullptr; }
}

// cuTensorMapEncodeTiled, fetched through the runtime (no link against the
// driver library); nullptr when the driver does not provide it.
using EncodeTiled = CUresult (*)(CUtensorMap *, CUtensorMapDataType, cuuint32_t, void *, const cuuint64_t *,
                                 const cuuint64_t *, const cuuint32_t *, const cuuint32_t *, CUtensorMapInterleave,
                                 CUtensorMapSwizzle, CUtensorMapL2promotion, CUtensorMapFloatOOBfill);

EncodeTiled tensor_map_encoder()
{
    static EncodeTiled fn = nullptr;
    static bool tried = false;
    if (!tried) {
        tried = true;
        void *ptr = nullptr;
        cudaDriverEntryPointQueryResult q;
        if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &ptr, 12000, cudaEnableDefault, &q) ==
                cudaSuccess &&
            q == cudaDriverEntryPointSuccess)
            fn = reinterpret_cast<EncodeTiled>(ptr);
        else
            cudaGetLastError();
    }
    return fn;
}

// The populations of one FP32 buffer as a tensor (x: nx, y: ny, plane: 13),
// boxes of the staged tile, zeros outside the lattice.
bool encode_lattice_map(lbm13_t h, const void *buf, CUtensorMap *m)
{
    const EncodeTiled fn = tensor_map_encoder();
    if (!fn) return false;
    const cuuint64_t dims[3] = {cuuint64_t(h->nx), cuuint64_t(h->ny), cuuint64_t(Q)};
    const cuuint64_t strides[2] = {cuuint64_t(h->pitch) * 4u, cuuint64_t(h->plane) * 4u};
    const cuuint32_t box[3] = {cuuint32_t(kTmaX), cuuint32_t(kTmaY), cuuint32_t(Q)};
    const cuuint32_t step[3] = {1, 1, 1};
    return fn(m, CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 3, const_cast<void *>(buf), dims, strides, box, step,
              CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE, CU_TENSOR_MAP_L2_PROMOTION_L2_128B,
              CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) == CUDA_SUCCESS;
}

// The same buffer ordered (x, plane, y) for the ring-staged strips: a box of
// box_x x 13 x kRingRows lands in shared memory as [row][plane][column].
bool encode_ring_map(lbm13_t h, const void *buf, CUtensorMap *m, int box_x)
{
    const EncodeTiled fn = tensor_map_encoder();
    if (!fn) return false;
    const cuuint64_t dims[3] = {cuuint64_t(h->nx), cuuint64_t(Q), cuuint64_t(h->ny)};
    const cuuint64_t strides[2] = {cuuint64_t(h->plane) * 4u, cuuint64_t(h->pitch) * 4u};
    const cuuint32_t box[3] = {cuuint32_t(box_x), cuuint32_t(Q), cuuint32_t(kRingRows)};
    const cuuint32_t step[3] = {1, 1, 1};
    return fn(m, CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 3, const_cast<void *>(buf), dims, strides, box, step,
              CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE, CU_TENSOR_MAP_L2_PROMOTION_L2_128B,
              CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) == CUDA_SUCCESS;
}

// The same buffer ordered (x, plane, y) in boxes of the paired steps' input
// tile: kPairInX x 13 x kPairInY lands in shared memory as [row][plane][column].
bool encode_pair_map(lbm13_t h, const void *buf, CUtensorMap *m)
{
    const EncodeTiled fn = tensor_map_encoder();
    if (!fn) return false;
    const cuuint64_t dims[3] = {cuuint64_t(h->nx), cuuint64_t(Q), cuuint64_t(h->ny)};
    const cuuint64_t strides[2] = {cuuint64_t(h->plane) * 4u, cuuint64_t(h->pitch) * 4u};
    const cuuint32_t box[3] = {cuuint32_t(kPairInX), cuuint32_t(Q), cuuint32_t(kPairInY)};
    const cuuint32_t step[3] = {1, 1, 1};
    return fn(m, CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 3, const_cast<void *>(buf), dims, strides, box, step,
              CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE, CU_TENSOR_MAP_L2_PROMOTION_L2_128B,
              CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) == CUDA_SUCCESS;
}

// Tensor maps of every lattice of an FP32 plan for both parities (lattices
// narrower than 64 columns or lower than the box keep global loads).
int plan_upload_maps(lbm13_plan_t p)
{
    std::vector<LatticeMaps> host(p->lats.size());
    p->ring_ok.assign(p->lats.size(), 0);
    for (size_t i = 0; i < p->lats.size(); ++i) {
        lbm13_t h = p->lats[i];
        std::memset(&host[i], 0, sizeof(LatticeMaps));
        const int cur = p->cur0[i];
        host[i].use = h->nx >= 64 && h->ny >= kTmaY && encode_lattice_map(h, h->buf[cur], &host[i].map[0]) &&
                      encode_lattice_map(h, h->buf[cur ^ 1], &host[i].map[1]);
        host[i].ring_use = h->nx >= 64 && h->ny >= kRingRows &&
                           encode_ring_map(h, h->buf[cur], &host[i].ring[0], Ring<64>::X) &&
                           encode_ring_map(h, h->buf[cur ^ 1], &host[i].ring[1], Ring<64>::X);
        host[i].ring32_use = h->nx >= 32 && h->ny >= kRingRows &&
                             encode_ring_map(h, h->buf[cur], &host[i].ring32[0], Ring<32>::X) &&
                             encode_ring_map(h, h->buf[cur ^ 1], &host[i].ring32[1], Ring<32>::X);
        p->ring_ok[i] = (host[i].ring_use ? 1 : 0) | (host[i].ring32_use ? 2 : 0);
    }
    const size_t bytes = host.size() * sizeof(LatticeMaps);
    const size_t cap_bytes = std::max(p->cap, host.size()) * sizeof(LatticeMaps);
    if (!p->maps || p->maps_bytes < bytes) {
        plan_free(p, p->maps);
        p->maps = plan_alloc(p, cap_bytes);
        p->maps_bytes = cap_bytes;
        if (!p->maps) return pfail(p, LBM13_ENOMEM, "allocator returned NULL for the plan's tensor maps");
    }
    if (!p->tma_err) {
        p->tma_err = static_cast<unsigned *>(plan_alloc(p, sizeof(unsigned)));
        if (!p->tma_err) return pfail(p, LBM13_ENOMEM, "allocator returned NULL for the plan's error word");
        cudaError_t e = cudaMemsetAsync(p->tma_err, 0, sizeof(unsigned), p->stream);
        if (e != cudaSuccess) return pfail(p, LBM13_ECUDA, std::string("plan error word: ") + cudaGetErrorString(e));
    }
    // pageable source: staged before the call returns, ordered on the plan's stream
    cudaError_t e = cudaMemcpyAsync(p->maps, host.data(), bytes, cudaMemcpyHostToDevice, p->stream);
    if (e != cudaSuccess) return pfail(p, LBM13_ECUDA, std::string("tensor map upload: ") + cudaGetErrorString(e));
    return LBM13_OK;
}

// Tensor maps of lattice i alone, into its slot (FP32 plans).
int plan_upload_map_one(lbm13_plan_t p, size_t i)
{
    lbm13_t h = p->lats[i];
    LatticeMaps m;
    std::memset(&m, 0, sizeof m);
    const int cur = p->cur0[i];
    m.use = h->nx >= 64 && h->ny >= kTmaY && encode_lattice_map(h, h->buf[cur], &m.map[0]) &&
            encode_lattice_map(h, h->buf[cur ^ 1], &m.map[1]);
    m.ring_use = h->nx >= 64 && h->ny >= kRingRows && encode_ring_map(h, h->buf[cur], &m.ring[0], Ring<64>::X) &&
                 encode_ring_map(h, h->buf[cur ^ 1], &m.ring[1], Ring<64>::X);
    m.ring32_use = h->nx >= 32 && h->ny >= kRingRows &&
                   encode_ring_map(h, h->buf[cur], &m.ring32[0], Ring<32>::X) &&
                   encode_ring_map(h, h->buf[cur ^ 1], &m.ring32[1], Ring<32>::X);
    if (p->ring_ok.size() <= i) p->ring_ok.resize(i + 1, 0);
    p->ring_ok[i] = (m.ring_use ? 1 : 0) | (m.ring32_use ? 2 : 0);
    cudaError_t e = cudaMemcpyAsync(static_cast<LatticeMaps *>(p->maps) + i, &m, sizeof m, cudaMemcpyHostToDevice,
                                    p->stream);
    if (e != cudaSuccess) return pfail(p, LBM13_ECUDA, std::string("tensor map upload: ") + cudaGetErrorString(e));
    return LBM13_OK;
}

template <typename T, typename C>
BatchDesc<T, C> batch_desc(lbm13_t h, int cur)
{
    BatchDesc<T, C> d;
    d.a[0] = step_args<T, C>(h, cur, coef_of<C>(h), walls_of<C>(h));
    d.a[1] = step_args<T, C>(h, cur ^ 1, coef_of<C>(h), walls_of<C>(h));
    d.force = h->force ? 1 : 0;
    d.tiles_x = (h->nx + 31) / 32;
    return d;
}

// The whole table (and, FP32, the tensor maps), every lattice taken at its
// current buffer: the plan's parity restarts at 0.
template <typename T, typename C>
int plan_upload_descs(lbm13_plan_t p)
{
    std::vector<BatchDesc<T, C>> host(p->lats.size());
    p->cur0.resize(p->lats.size());
    for (size_t i = 0; i < p->lats.size(); ++i) {
        lbm13_t h = p->lats[i];
        host[i] = batch_desc<T, C>(h, h->cur);
        p->cur0[i] = h->cur;
    }
    const size_t bytes = host.size() * sizeof(BatchDesc<T, C>);
    p->cap = std::max(p->cap, host.size());
    const size_t cap_bytes = p->cap * sizeof(BatchDesc<T, C>);
    if (!p->desc || p->desc_bytes < bytes) {
        plan_free(p, p->desc);
        p->desc = plan_alloc(p, cap_bytes);
        p->desc_bytes = cap_bytes;
        if (!p->desc) return pfail(p, LBM13_ENOMEM, "allocator returned NULL for the plan table");
    }
    // pageable source: staged before the call returns, ordered on the plan's stream
    cudaError_t e = cudaMemcpyAsync(p->desc, host.data(), bytes, cudaMemcpyHostToDevice, p->stream);
    if (e != cudaSuccess) return pfail(p, LBM13_ECUDA, std::string("plan table upload: ") + cudaGetErrorString(e));
    if (sizeof(T) == 4) {
        const int rc = plan_upload_maps(p);
        if (rc != LBM13_OK) return rc;
    }
    p->parity = 0;
    plan_drop_graphs(p);
    return LBM13_OK;
}

// Work list for tiles of 32 columns x groups * BY * R rows, each packed as
// (tile row << 16) | tile column (both below 2^15 within the lattice limits),
// in one of three orders: 0 lattice by lattice, 1 round robin across
// lattices, 2 largest lattice first.  The ring-staged strips of a lattice with
// ring maps step only the nodes two links or more from every edge; its edge
// nodes (ring_edge_count, Ring<W>::EdgeNodes per item) come as items packed
// -1 - item, ahead of its strips, so that their latency-bound global loads run
// beside streaming strips.
bool plan_is_ring(const lbm13_plan *p) { return p->R == 0 && (p->BY == 8 || p->BY == 4); }
// Strip width of the ring-staged shapes: eight warps take 64 columns, four 32.
int plan_ring_width(const lbm13_plan *p) { return p->BY == 8 ? 64 : 32; }

int plan_build_work(lbm13_plan_t p)
{
    // ring tiles: strips of 64 or 32 columns x groups 4-row groups
    const bool ring = plan_is_ring(p);
    const int rows = ring ? kRingRows * p->groups : p->R * p->BY * p->groups;
    const int cols = ring ? plan_ring_width(p) : 32;
    const size_t L = p->lats.size();
    std::vector<std::vector<int2>> per(L);
    for (size_t i = 0; i < L; ++i) {
        lbm13_t h = p->lats[i];
        const int tx = (h->nx + cols - 1) / cols, ty = (h->ny + rows - 1) / rows;
        per[i].reserve(size_t(tx) * ty);
        const unsigned bit = plan_ring_width(p) == 64 ? 1u : 2u;
        if (ring && i < p->ring_ok.size() && (p->ring_ok[i] & bit)) {
            const long long per_item = plan_ring_width(p) == 64 ? Ring<64>::EdgeNodes : Ring<32>::EdgeNodes;
            const long long items = (ring_edge_count(h->nx, h->ny) + per_item - 1) / per_item;
            for (long long e = 0; e < items; ++e) per[i].push_back(make_int2(int(i), int(-1 - e)));
        }
        for (int y = 0; y < ty; ++y)
            for (int x = 0; x < tx; ++x) per[i].push_back(make_int2(int(i), (y << 16) | x));
    }
    std::vector<int2> work;
    std::vector<size_t> idx(L);
    for (size_t i = 0; i < L; ++i) idx[i] = i;
    if (p->order == 2)
        std::stable_sort(idx.begin(), idx.end(), [&](size_t a, size_t b) { return per[a].size() > per[b].size(); });
    if (p->order == 1) {
        size_t most = 0;
        for (auto &v : per) most = std::max(most, v.size());
        for (size_t k = 0; k < most; ++k)
            for (size_t i = 0; i < L; ++i)
                if (k < per[i].size()) work.push_back(per[i][k]);
    } else {
        for (size_t i : idx) work.insert(work.end(), per[i].begin(), per[i].end());
    }
    p->ntiles = int(work.size());
    const size_t bytes = std::max<size_t>(work.size(), 1) * sizeof(int2);
    if (!p->work || p->work_bytes < bytes) {
        // the old list may still be read by launches in flight on the plan's
        // stream: the allocator's free is stream-ordered (cudaFree waits)
        plan_free(p, p->work);
        p->work = plan_alloc(p, bytes + bytes / 2);
        p->work_bytes = bytes + bytes / 2;
        if (!p->work) return pfail(p, LBM13_ENOMEM, "allocator returned NULL for the work list");
    }
    cudaError_t e = cudaMemcpyAsync(p->work, work.data(), work.size() * sizeof(int2), cudaMemcpyHostToDevice, p->stream);
    if (e != cudaSuccess) return pfail(p, LBM13_ECUDA, std::string("work list upload: ") + cudaGetErrorString(e));
    p->grid = p->ctas <= 0 ? p->ntiles : std::min(p->ntiles, p->sms * p->ctas);
    if (p->grid < 1) p->grid = 1;
    plan_drop_graphs(p);
    return LBM13_OK;
}

cudaError_t plan_launch(lbm13_plan_t p, int parity, cudaStream_t s)
{
    if (plan_is_ring(p)) {
        if (p->precision == LBM13_FP64 || !p->maps || !p->tma_err) return cudaErrorInvalidValue;
        return launch_batch_ring(static_cast<const BatchDesc<float, float> *>(p->desc),
                                 static_cast<const LatticeMaps *>(p->maps), static_cast<const int2 *>(p->work),
                                 p->ntiles, parity, p->groups, plan_ring_width(p), p->tma_err, s);
    }
    if (p->precision != LBM13_FP64 && p->R == 4 && p->BY == 4 && p->grid >= p->ntiles && p->maps && p->tma_err)
        return launch_batch_tma(static_cast<const BatchDesc<float, float> *>(p->desc),
                                static_cast<const LatticeMaps *>(p->maps), static_cast<const int2 *>(p->work),
                                p->ntiles, parity, p->groups, p->tma_err, s);
    if (p->precision == LBM13_FP64) {
        const auto *d = static_cast<const BatchDesc<double, double> *>(p->desc);
        return launch_batch<double, double>(d, static_cast<const int2 *>(p->work), p->ntiles, parity, p->R, p->BY,
                                            p->groups, p->grid, s);
    }
    const auto *d = static_cast<const BatchDesc<float, float> *>(p->desc);
    return launch_batch<float, float>(d, static_cast<const int2 *>(p->work), p->ntiles, parity, p->R, p->BY,
                                      p->groups, p->grid, s);
}

// Re-upload the table when a lattice was stepped or reset outside the plan.
int plan_sync_parity(lbm13_plan_t p)
{
    for (size_t i = 0; i < p->lats.size(); ++i)
        if (p->lats[i]->cur != (p->cur0[i] ^ p->parity))
            return p->precision == LBM13_FP64 ? plan_upload_descs<double, double>(p) : plan_upload_descs<float, float>(p);
    return LBM13_OK;
}

void plan_advance(lbm13_plan_t p, long long n)
{
    for (lbm13_t h : p->lats) {
        h->cur ^= int(n & 1);
        h->t += n;
    }
    p->parity ^= int(n & 1);
}

int plan_steps(lbm13_plan_t p, long long n)
{
    int rc = plan_sync_parity(p);
    if (rc != LBM13_OK) return rc;
    if (n >= kGraphSteps) {
        if (!p->gexec[p->parity]) {
            cudaError_t e = cudaSuccess;
            if (!p->cap_stream) e = cudaStreamCreateWithFlags(&p->cap_stream, cudaStreamNonBlocking);
            if (e == cudaSuccess) e = cudaStreamBeginCapture(p->cap_stream, cudaStreamCaptureModeThreadLocal);
            if (e != cudaSuccess) return pfail(p, LBM13_ECUDA, std::string("plan graph capture: ") + cudaGetErrorString(e));
            cudaError_t le = cudaSuccess;
            for (long long i = 0; i < kGraphSteps && le == cudaSuccess; ++i)
                le = plan_launch(p, p->parity ^ int(i & 1), p->cap_stream);
            cudaGraph_t g = nullptr;
            e = cudaStreamEndCapture(p->cap_stream, &g);
            if (le != cudaSuccess) e = le;
            if (e == cudaSuccess) e = cudaGraphInstantiate(&p->gexec[p->parity], g, 0);
            if (g) cudaGraphDestroy(g);
            if (e != cudaSuccess) return pfail(p, LBM13_ECUDA, std::string("plan graph: ") + cudaGetErrorString(e));
        }
        for (; n >= kGraphSteps; n -= kGraphSteps) {
            cudaError_t e = cudaGraphLaunch(p->gexec[p->parity], p->stream);
            if (e != cudaSuccess) return pfail(p, LBM13_ECUDA, std::string("cudaGraphLaunch (plan): ") + cudaGetErrorString(e));
            plan_advance(p, kGraphSteps);
        }
    }
    for (long long i = 0; i < n; ++i) {
        cudaError_t e = plan_launch(p, p->parity, p->stream);
        if (e != cudaSuccess) return pfail(p, LBM13_ECUDA, std::string("batched step launch: ") + cudaGetErrorString(e));
        plan_advance(p, 1);
    }
    return LBM13_OK;
}

// Make the plan's stream wait for the work already issued on `from`.
int plan_order_after(lbm13_plan_t p, cudaStream_t from, cudaStream_t to)
{
    cudaError_t e = cudaSuccess;
    if (!p->order_ev) e = cudaEventCreateWithFlags(&p->order_ev, cudaEventDisableTiming);
    if (e == cudaSuccess) e = cudaEventRecord(p->order_ev, from);
    if (e == cudaSuccess) e = cudaStreamWaitEvent(to, p->order_ev, 0);
    if (e != cudaSuccess) return pfail(p, LBM13_ECUDA, std::string("stream ordering: ") + cudaGetErrorString(e));
    return LBM13_OK;
}

template <typename T, typename C>
int plan_add_one(lbm13_plan_t p, lbm13_t h)
{
    const size_t i = p->lats.size();
    p->lats.push_back(h);
    // the plan's next launch reads buffer cur0 ^ parity of every lattice
    p->cur0.push_back(h->cur ^ p->parity);
    p->nodes += (long long)h->nx * h->ny;
    if (i >= p->cap) {
        // grow the table (and maps) to twice the lattices: re-upload every
        // lattice's entry at its current buffer (plan parity restarts at 0)
        p->cap = std::max<size_t>(2 * (i + 1), 8);
        plan_free(p, p->desc);
        p->desc = nullptr;
        p->desc_bytes = 0;
        plan_free(p, p->maps);
        p->maps = nullptr;
        p->maps_bytes = 0;
        return plan_upload_descs<T, C>(p);
    }
    const BatchDesc<T, C> d = batch_desc<T, C>(h, p->cur0[i]);
    cudaError_t e = cudaMemcpyAsync(static_cast<BatchDesc<T, C> *>(p->desc) + i, &d, sizeof d,
                                    cudaMemcpyHostToDevice, p->stream);
    if (e != cudaSuccess) return pfail(p, LBM13_ECUDA, std::string("plan table entry: ") + cudaGetErrorString(e));
    if (sizeof(T) == 4 && p->maps) return plan_upload_map_one(p, i);
    return LBM13_OK;
}

// Lattice i leaves: the last lattice takes its slot (entry and maps copied on
// the plan's stream, after the launches that still read them).
template <typename T, typename C>
int plan_remove_one(lbm13_plan_t p, size_t i)
{
    const size_t last = p->lats.size() - 1;
    p->nodes -= (long long)p->lats[i]->nx * p->lats[i]->ny;
    if (i != last) {
        p->lats[i] = p->lats[last];
        p->cur0[i] = p->cur0[last];
        if (last < p->ring_ok.size()) p->ring_ok[i] = p->ring_ok[last];
        auto *d = static_cast<BatchDesc<T, C> *>(p->desc);
        cudaError_t e = cudaMemcpyAsync(d + i, d + last, sizeof(BatchDesc<T, C>), cudaMemcpyDeviceToDevice, p->stream);
        if (e == cudaSuccess && sizeof(T) == 4 && p->maps) {
            auto *m = static_cast<LatticeMaps *>(p->maps);
            e = cudaMemcpyAsync(m + i, m + last, sizeof(LatticeMaps), cudaMemcpyDeviceToDevice, p->stream);
        }
        if (e != cudaSuccess) return pfail(p, LBM13_ECUDA, std::string("plan table move: ") + cudaGetErrorString(e));
    }
    p->lats.pop_back();
    p->cur0.pop_back();
    if (p->ring_ok.size() > p->lats.size()) p->ring_ok.resize(p->lats.size());
    return LBM13_OK;
}

} // namespace

extern "C" {

int lbm13_plan_create(const lbm13_t *lattices, int count, const lbm13_allocator *alloc, void *stream,
                      lbm13_plan_t *out)
{
    if (!out) return pfail(nullptr, LBM13_EINVAL, "out is NULL");
    *out = nullptr;
    if (!lattices || count <= 0) return pfail(nullptr, LBM13_EINVAL, "empty lattice list");
    if (alloc && (!alloc->alloc || !alloc->free)) return pfail(nullptr, LBM13_EINVAL, "allocator without alloc/free");
    for (int i = 0; i < count; ++i) {
        if (!lattices[i]) return pfail(nullptr, LBM13_EINVAL, "NULL lattice in the list");
        if (lattices[i]->precision != lattices[0]->precision || lattices[i]->device != lattices[0]->device)
            return pfail(nullptr, LBM13_EINVAL, "lattices of one plan must share precision and device");
        for (int k = 0; k < i; ++k)
            if (lattices[k] == lattices[i]) return pfail(nullptr, LBM13_EINVAL, "a lattice appears twice");
    }
    lbm13_plan_t p = new lbm13_plan();
    p->lats.assign(lattices, lattices + count);
    p->precision = lattices[0]->precision;
    p->device = lattices[0]->device;
    p->stream = static_cast<cudaStream_t>(stream);
    if (alloc) { p->alloc = *alloc; p->has_alloc = true; }
    DeviceGuard g(p->device);
    cudaDeviceProp prop;
    if (cudaGetDeviceProperties(&prop, p->device) != cudaSuccess) {
        delete p;
        return pfail(nullptr, LBM13_ECUDA, "cudaGetDeviceProperties");
    }
    p->sms = prop.multiProcessorCount;
    for (lbm13_t h : p->lats) p->nodes += (long long)h->nx * h->ny;
    // the lattices' own streams must be idle before the plan takes over
    for (lbm13_t h : p->lats) cudaStreamSynchronize(h->stream);
    int rc = p->precision == LBM13_FP64 ? plan_upload_descs<double, double>(p) : plan_upload_descs<float, float>(p);
    if (rc == LBM13_OK) rc = plan_build_work(p);
    if (rc != LBM13_OK) {
        lbm13_plan_destroy(p);
        return rc;
    }
    *out = p;
    return LBM13_OK;
}

void lbm13_plan_destroy(lbm13_plan_t p)
{
    if (!p) return;
    DeviceGuard g(p->device);
    cudaStreamSynchronize(p->stream);
    plan_drop_graphs(p);
    if (p->cap_stream) cudaStreamDestroy(p->cap_stream);
    plan_free(p, p->desc);
    plan_free(p, p->work);
    plan_free(p, p->maps);
    plan_free(p, p->tma_err);
    plan_free(p, p->res_dev);
    if (p->order_ev) cudaEventDestroy(p->order_ev);
    delete p;
}

int lbm13_plan_add(lbm13_plan_t p, lbm13_t h)
{
    Range range_("lbm13_plan_add");
    if (!p || !h) return pfail(p, LBM13_EINVAL, "NULL plan or lattice");
    if (h->precision != p->precision || h->device != p->device)
        return pfail(p, LBM13_EINVAL, "the lattice's precision or device differs from the plan's");
    for (lbm13_t q : p->lats)
        if (q == h) return pfail(p, LBM13_EINVAL, "the lattice is already in the plan");
    DeviceGuard g(p->device);
    // work issued on the lattice's own stream (creation, initial state) comes first
    int rc = plan_order_after(p, h->stream, p->stream);
    if (rc == LBM13_OK)
        rc = p->precision == LBM13_FP64 ? plan_add_one<double, double>(p, h) : plan_add_one<float, float>(p, h);
    if (rc == LBM13_OK) rc = plan_build_work(p);
    return rc;
}

int lbm13_plan_remove(lbm13_plan_t p, lbm13_t h)
{
    Range range_("lbm13_plan_remove");
    if (!p || !h) return pfail(p, LBM13_EINVAL, "NULL plan or lattice");
    size_t i = 0;
    while (i < p->lats.size() && p->lats[i] != h) ++i;
    if (i == p->lats.size()) return pfail(p, LBM13_EINVAL, "the lattice is not in the plan");
    if (p->lats.size() == 1) return pfail(p, LBM13_EINVAL, "a plan keeps at least one lattice (destroy it instead)");
    DeviceGuard g(p->device);
    int rc = p->precision == LBM13_FP64 ? plan_remove_one<double, double>(p, i) : plan_remove_one<float, float>(p, i);
    // the lattice's own stream waits for the plan's launches that step it
    if (rc == LBM13_OK) rc = plan_order_after(p, p->stream, h->stream);
    if (rc == LBM13_OK) rc = plan_build_work(p);
    return rc;
}

const char *lbm13_plan_last_error(lbm13_plan_t p) { return p ? p->err.c_str() : g_err.c_str(); }

int lbm13_plan_set_config(lbm13_plan_t p, int R, int BY, int ctas_per_sm, int order, int groups)
{
    if (!p) return pfail(nullptr, LBM13_EINVAL, "NULL plan");
    if (!batch_shape_supported(R, BY) || order < 0 || order > 2 || ctas_per_sm < 0 || ctas_per_sm > 64 ||
        groups < 1 || groups > 64)
        return pfail(p, LBM13_EINVAL, "unsupported tile shape, order, CTA count or row groups");
    if (R == 0 && p->precision == LBM13_FP64)
        return pfail(p, LBM13_EINVAL, "the ring-staged tile shapes (R = 0, BY = 8 or 4) are FP32 only");
    DeviceGuard g(p->device);
    p->R = R;
    p->BY = BY;
    p->ctas = ctas_per_sm;
    p->order = order;
    p->groups = groups;
    return plan_build_work(p);
}

int lbm13_plan_tma_check(lbm13_plan_t p, double timeout_s, int withhold, int *timed_out)
{
    if (!p || !timed_out || !(timeout_s >= 1e-3 && timeout_s <= 2.0))
        return pfail(p, LBM13_EINVAL, "NULL argument or timeout_s outside [1e-3, 2]");
    const bool ring = plan_is_ring(p);
    if (p->precision == LBM13_FP64 || !p->maps || !p->tma_err ||
        !(ring || (p->R == 4 && p->BY == 4 && p->grid >= p->ntiles)))
        return pfail(p, LBM13_EINVAL,
                     "the plan is not on staged FP32 tiles (R = 4, BY = 4, one CTA per tile; or the ring, R = 0, BY = 8 or 4)");
    DeviceGuard g(p->device);
    int rc = plan_sync_parity(p);
    if (rc != LBM13_OK) return rc;
    unsigned word = 0;
    const auto *descs = static_cast<const BatchDesc<float, float> *>(p->desc);
    const auto *maps = static_cast<const LatticeMaps *>(p->maps);
    const auto *work = static_cast<const int2 *>(p->work);
    const unsigned long long wait_ns = (unsigned long long)(timeout_s * 1e9);
    cudaError_t e = ring ? launch_batch_ring(descs, maps, work, p->ntiles, p->parity, p->groups, plan_ring_width(p),
                                             p->tma_err, p->stream, withhold ? 0 : 1, wait_ns)
                         : launch_batch_tma(descs, maps, work, p->ntiles, p->parity, p->groups, p->tma_err, p->stream,
                                            withhold ? 0 : 1, wait_ns);
    if (e == cudaSuccess) e = cudaStreamSynchronize(p->stream);
    if (e == cudaSuccess) e = cudaMemcpy(&word, p->tma_err, sizeof word, cudaMemcpyDeviceToHost);
    if (e == cudaSuccess) e = cudaMemset(p->tma_err, 0, sizeof word);
    if (e != cudaSuccess) return pfail(p, LBM13_ECUDA, std::string("staged tile check: ") + cudaGetErrorString(e));
    *timed_out = word != 0u;
    return LBM13_OK;
}

int lbm13_plan_config(lbm13_plan_t p, int64_t out[9])
{
    if (!p || !out) return pfail(p, LBM13_EINVAL, "NULL argument");
    out[0] = p->R;
    out[1] = p->BY;
    out[2] = p->ctas;
    out[3] = p->order;
    out[4] = p->ntiles;
    out[5] = p->grid;
    out[6] = p->nodes;
    out[7] = p->tried;
    out[8] = p->groups;
    return LBM13_OK;
}

int lbm13_plan_step(lbm13_plan_t p, int64_t n)
{
    Range range_("lbm13_plan_step");
    if (!p || n < 0) return pfail(p, LBM13_EINVAL, "NULL plan or negative step count");
    DeviceGuard g(p->device);
    return plan_steps(p, n);
}

int lbm13_plan_residual(lbm13_plan_t p, double *out)
{
    Range range_("lbm13_plan_residual");
    if (!p || !out) return pfail(p, LBM13_EINVAL, "NULL argument");
    DeviceGuard g(p->device);
    const size_t bytes = p->lats.size() * 16 * sizeof(double);
    if (!p->res_dev || p->res_cap < p->lats.size()) {
        plan_free(p, p->res_dev);
        p->res_cap = std::max(p->cap, p->lats.size());
        p->res_dev = static_cast<double *>(plan_alloc(p, p->res_cap * 16 * sizeof(double)));
        if (!p->res_dev) return pfail(p, LBM13_ENOMEM, "allocator returned NULL for the plan's residual buffer");
    }
    for (size_t i = 0; i < p->lats.size(); ++i) {
        lbm13_t h = p->lats[i];
        int rc = ensure_reduce(h);
        if (rc != LBM13_OK) return pfail(p, rc, h->err);
        cudaError_t e = launch_residual(h, p->res_dev + 16 * i, p->stream);
        if (e != cudaSuccess) return pfail(p, LBM13_ECUDA, std::string("plan reduction launch: ") + cudaGetErrorString(e));
    }
    cudaError_t e = cudaMemcpyAsync(out, p->res_dev, bytes, cudaMemcpyDeviceToHost, p->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(p->stream);
    if (e != cudaSuccess) return pfail(p, LBM13_ECUDA, std::string("plan residual download: ") + cudaGetErrorString(e));
    if (p->tma_err) {
        unsigned word = 0;
        e = cudaMemcpy(&word, p->tma_err, sizeof word, cudaMemcpyDeviceToHost);
        if (e == cudaSuccess && word) e = cudaMemset(p->tma_err, 0, sizeof word);
        if (e != cudaSuccess) return pfail(p, LBM13_ECUDA, std::string("plan error word: ") + cudaGetErrorString(e));
        if (word) return pfail(p, LBM13_ETIMEOUT, "a staged tile's tensor copy did not complete within 1 s");
    }
    bool bad = false;
    for (size_t i = 0; i < p->lats.size(); ++i) {
        p->lats[i]->have_snap = 1;
        p->lats[i]->snap_t = p->lats[i]->t;
        bad = bad || out[16 * i + LBM13_R_NONFINITE] > 0.0;
    }
    return bad ? pfail(p, LBM13_EDIVERGED, "non-finite populations in a lattice of the plan") : LBM13_OK;
}

int lbm13_plan_tune(lbm13_plan_t p, int steps_per_candidate, double *best_ms_per_step)
{
    Range range_("lbm13_plan_tune");
    if (!p || steps_per_candidate < 1) return pfail(p, LBM13_EINVAL, "NULL plan or steps_per_candidate < 1");
    DeviceGuard g(p->device);
    struct Cand {
        int R, BY, ctas, groups, order;
    };
    std::vector<Cand> cands;
    static const int shapes[][2] = {{1, 4}, {2, 4}, {4, 4}, {2, 2}, {1, 8}};
    static const int ctas[] = {0, 4, 8, 16};
    static const int groups[] = {1, 4, 16};
    for (const auto &sh : shapes)
        for (int c : ctas)
            for (int gr : groups)
                for (int o = 0; o < 3; ++o) cands.push_back({sh[0], sh[1], c, gr, o});
    // ring-staged strips (FP32), 64 and 32 columns wide: one block per strip
    // segment of 4 groups rows
    static const int ring_groups[] = {4, 8, 16, 32};
    if (p->precision != LBM13_FP64)
        for (int by : {8, 4})
            for (int gr : ring_groups)
                for (int o = 0; o < 3; ++o) cands.push_back({0, by, 0, gr, o});
    cudaEvent_t e0, e1;
    if (cudaEventCreate(&e0) != cudaSuccess || cudaEventCreate(&e1) != cudaSuccess)
        return pfail(p, LBM13_ECUDA, "cudaEventCreate");
    double best = 1e300;
    Cand b = {p->R, p->BY, p->ctas, p->groups, p->order};
    int rc = LBM13_OK;
    p->tried = 0;
    for (const Cand &c : cands) {
        p->R = c.R;
        p->BY = c.BY;
        p->ctas = c.ctas;
        p->order = c.order;
        p->groups = c.groups;
        if ((rc = plan_build_work(p)) != LBM13_OK) break;
        if ((rc = plan_steps(p, 1)) != LBM13_OK) break;  // warm-up
        cudaEventRecord(e0, p->stream);
        if ((rc = plan_steps(p, steps_per_candidate)) != LBM13_OK) break;
        cudaEventRecord(e1, p->stream);
        if (cudaEventSynchronize(e1) != cudaSuccess) { rc = pfail(p, LBM13_ECUDA, "tuning event"); break; }
        float ms = 0.f;
        cudaEventElapsedTime(&ms, e0, e1);
        const double per = double(ms) / steps_per_candidate;
        ++p->tried;
        if (per < best) { best = per; b = c; }
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    if (rc != LBM13_OK) return rc;
    p->R = b.R;
    p->BY = b.BY;
    p->ctas = b.ctas;
    p->order = b.order;
    p->groups = b.groups;
    if ((rc = plan_build_work(p)) != LBM13_OK) return rc;
    if (best_ms_per_step) *best_ms_per_step = best;
    return LBM13_OK;
}

} // extern "C"
