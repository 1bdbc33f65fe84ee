// C-ABI layer: argument checks, handle (tables, groups, workspace), dispatch of the
// split-step passes, status word.  Declarations and contracts: include/gpe.h.
#include <cmath>
#include <cstdarg>
#include <cstdio>
#include <cstring>
#include <algorithm>
#include <atomic>
#include <map>
#include <new>
#include <string>
#include <tuple>
#include <vector>

#include <cudaTypedefs.h>
#include <nvtx3/nvToolsExt.h>

#include "adjoint.h"
#include "gpe.h"
#include "internal.h"
#include "obs.h"

using namespace gpe;

namespace {

thread_local std::string g_err;

gpe_status fail(gpe_status s, const char* fmt, ...) {
    char buf[512];
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(buf, sizeof(buf), fmt, ap);
    va_end(ap);
    g_err = buf;
    return s;
}

#define GPE_CK(call)                                                                      \
    do {                                                                                  \
        cudaError_t e_ = (call);                                                          \
        if (e_ != cudaSuccess) return fail(GPE_ECUDA, "%s: %s", #call, cudaGetErrorString(e_)); \
    } while (0)

bool is_pow2(int n) { return n > 0 && (n & (n - 1)) == 0; }

std::atomic<int64_t> g_launches{0};

// Allocation-failure test hook: number of device allocations still allowed to succeed
// before one fails (-1: off).
std::atomic<int64_t> g_alloc_fail_after{-1};
std::atomic<int> g_table_tmem{1};   // gpe_debug_table_memory

constexpr int kProfKinds = 6;

struct Profiler {
    bool on = false;
    std::vector<cudaEvent_t> pool;
    std::vector<std::pair<int, std::pair<cudaEvent_t, cudaEvent_t>>> open;
    size_t used = 0;
    cudaEvent_t get() {
        if (used == pool.size()) {
            cudaEvent_t e;
            cudaEventCreate(&e);
            pool.push_back(e);
        }
        return pool[used++];
    }
};

}  // namespace

void gpe::set_last_error(const char* msg) { g_err = msg ? msg : ""; }

bool gpe::tables_in_tmem() { return g_table_tmem.load() != 0; }

cudaError_t gpe::device_malloc(void** p, size_t bytes) {
    int64_t left = g_alloc_fail_after.load();
    while (left >= 0) {
        // the hook counts down once per allocation; at zero this one fails and it switches off
        if (g_alloc_fail_after.compare_exchange_weak(left, left - 1)) {
            if (left == 0) {
                *p = nullptr;
                return cudaErrorMemoryAllocation;
            }
            break;
        }
    }
    return cudaMalloc(p, bytes);
}

namespace {

PFN_cuTensorMapEncodeTiled_v12000 tensor_map_encoder() {
    static PFN_cuTensorMapEncodeTiled_v12000 fn = nullptr;
    static bool tried = false;
    if (!tried) {
        tried = true;
        void* p = nullptr;
        cudaDriverEntryPointQueryResult q;
        if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault, &q) ==
                cudaSuccess &&
            q == cudaDriverEntryPointSuccess)
            fn = reinterpret_cast<PFN_cuTensorMapEncodeTiled_v12000>(p);
        else
            cudaGetLastError();
    }
    return fn;
}

}  // namespace

// Tensor maps over a contiguous group: y pencils through a 2D view {2 nx, ntraj 3 nz ny}
// of the whole batch, z pencils through a 3D view {2 nx, ny, nz 3 ntraj}; boxes are
// COLS complex columns wide and min(n, 256) points long.
bool gpe::encode_maps(CUtensorMap* map_y, CUtensorMap* map_z, const Group& g, void* base, int ntraj, int eb,
                      int cols_y, int cols_z) {
    PFN_cuTensorMapEncodeTiled_v12000 enc = tensor_map_encoder();
    if (!enc || g.ndim < 2) return false;
    const CUtensorMapDataType dt = eb == 4 ? CU_TENSOR_MAP_DATA_TYPE_FLOAT32 : CU_TENSOR_MAP_DATA_TYPE_FLOAT64;
    const cuuint64_t nx = g.n[0], ny = g.n[1], nz = g.n[2];
    const cuuint32_t es[3] = {1, 1, 1};
    {
        const cuuint64_t dims[2] = {2 * nx, (cuuint64_t)ntraj * 3 * nz * ny};
        const cuuint64_t strides[1] = {2 * nx * (cuuint64_t)eb};
        const cuuint32_t box[2] = {(cuuint32_t)(2 * cols_y), (cuuint32_t)(ny < 256 ? ny : 256)};
        if (enc(map_y, dt, 2, base, dims, strides, box, es, CU_TENSOR_MAP_INTERLEAVE_NONE,
                CU_TENSOR_MAP_SWIZZLE_NONE, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
                CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) != CUDA_SUCCESS)
            return false;
    }
    if (g.ndim == 3) {
        const cuuint64_t dims[3] = {2 * nx, ny, nz * 3 * (cuuint64_t)ntraj};
        const cuuint64_t strides[2] = {2 * nx * (cuuint64_t)eb, 2 * nx * ny * (cuuint64_t)eb};
        const cuuint32_t box[3] = {(cuuint32_t)(2 * cols_z), 1, (cuuint32_t)(nz < 256 ? nz : 256)};
        if (enc(map_z, dt, 3, base, dims, strides, box, es, CU_TENSOR_MAP_INTERLEAVE_NONE,
                CU_TENSOR_MAP_SWIZZLE_NONE, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
                CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) != CUDA_SUCCESS)
            return false;
    }
    return true;
}

bool gpe::encode_group_maps(Group& g, int eb) {
    return encode_maps(&g.map_y, &g.map_z, g, g.hptrs[0], g.ntraj, eb, g.cols[1], g.ndim == 3 ? g.cols[2] : g.cols[1]);
}

struct gpe_batch {
    gpe_dtype dtype;
    gpe_params p;
    std::vector<double> knots;
    double* d_knots = nullptr;
    std::vector<gpe_traj> trajs;
    std::vector<Group> groups;
    int64_t step = 0;
    int integrator = 0;               // GPE_INTEGRATOR_PAPER or GPE_INTEGRATOR_ROTATION
    bool autotune = true;             // time the column-pass tile widths on the first step
    int64_t traj_base = 0;            // added to batch indices in the noise counter
    uint32_t wait_first = 0;          // first copy wait's poll limit of the passes (0: default, else 1 + limit)
    int* d_status = nullptr;
    int device = 0;
    std::vector<void*> allocs;
    ObsWork obs;
    Profiler prof;
    // concurrency across shape groups and trajectory lanes (one stream per work item of
    // run_steps, created on demand), and CUDA-graph replay of whole step sequences
    int lanes_req = -1;               // gpe_batch_set_lanes: -1 the default, else lanes per 2D/3D group
    std::vector<cudaStream_t> gstream;
    cudaEvent_t ev_fork = nullptr;
    std::vector<cudaEvent_t> ev_join;
    cudaStream_t cap_stream = nullptr;
    bool graph_mode = false;
    struct GraphEntry {
        cudaGraphExec_t exec;
        int64_t launches;
    };
    std::map<int64_t, GraphEntry> graphs;
    // adjoint / loss workspace (allocated on first use)
    void* adj_phi = nullptr;        // ntraj x 3 x sites
    void* adj_W = nullptr;          // ntraj x sites
    void** adj_ptrs = nullptr;      // 3 x ntraj pointer tables
    void* adj_phc[3] = {};          // per strided axis: conjugated half-step phase table
    double* adj_part = nullptr;     // partial sums
    int64_t adj_nparts = 0;
};

namespace {

// NVTX range names of the kernel classes (host-side ranges around each launch sequence,
// for timeline tools; they cost a pointer test when no tool is attached).
constexpr const char* kNvtxNames[kProfKinds] = {"gpe.xpass", "gpe.strided_pass", "gpe.resident1d",
                                                "gpe.noise", "gpe.observables", "gpe.adjoint"};

// Brackets one launch (or launch sequence) of class ``kind`` with an NVTX range and, when
// profiling, with events.
struct ProfScope {
    gpe_batch* b;
    int kind;
    cudaStream_t s;
    cudaEvent_t e1 = nullptr;
    ProfScope(gpe_batch* b_, int kind_, cudaStream_t s_, int64_t nlaunch) : b(b_), kind(kind_), s(s_) {
        g_launches += nlaunch;
        nvtxRangePushA(kNvtxNames[kind]);
        if (b->prof.on) {
            cudaEvent_t e0 = b->prof.get();
            e1 = b->prof.get();
            cudaEventRecord(e0, s);
            b->prof.open.push_back({kind, {e0, e1}});
        }
    }
    ~ProfScope() {
        if (e1) cudaEventRecord(e1, s);
        nvtxRangePop();
    }
};

}  // namespace

namespace {

// Kinetic phase tables exp(-i tau k^2/2) / n for tau = dt and dt/2, computed in FP64.
// Table entry from an FP64 complex value c = m e^{i phi}.  FP32 keeps the three-shear form
// of the rotation (common.cuh): phi reduced by a multiple j of pi into [-pi/2, pi/2] (with a
// margin of 1e-12 so angles that are exactly +-pi/2 keep j = 0), then (-tan(phi/2), sin(phi),
// (-1)^j m, 0), each rounded once from FP64.
template <typename T> twel<T> tw_entry(double re, double im);
template <> float4 tw_entry<float>(double re, double im) {
    const double pi = 3.14159265358979323846, half_pi = 1.57079632679489661923;
    const double m = std::hypot(re, im);
    double phi = std::atan2(im, re);
    double s = m;
    if (phi > half_pi + 1e-12) {
        phi -= pi;
        s = -m;
    } else if (phi < -half_pi - 1e-12) {
        phi += pi;
        s = -m;
    }
    return make_float4((float)(-std::tan(0.5 * phi)), (float)std::sin(phi), (float)s, 0.0f);
}
template <> double2 tw_entry<double>(double re, double im) { return make_double2(re, im); }

// The conjugate of a table entry: FP32 (p, u, s) -> (-p, -u, s) (rotation by minus the
// reduced angle, same reduction sign), FP64 (re, im) -> (re, -im); exact.
float4 conj_entry(float4 e) { return make_float4(-e.x, -e.y, e.z, e.w); }
double2 conj_entry(double2 e) { return make_double2(e.x, -e.y); }

template <typename T>
void phase_tables_host(int n, double dx, double dt, std::vector<twel<T>>& pf, std::vector<twel<T>>& ph) {
    pf.resize(n);
    ph.resize(n);
    const double two_pi = 6.283185307179586476925286766559;
    for (int i = 0; i < n; ++i) {
        const int j = (i < n / 2) ? i : i - n;
        const double k = two_pi * (double)j / ((double)n * dx);
        const double a_full = 0.5 * dt * k * k, a_half = 0.25 * dt * k * k;
        pf[i] = tw_entry<T>(std::cos(a_full) / n, -std::sin(a_full) / n);
        ph[i] = tw_entry<T>(std::cos(a_half) / n, -std::sin(a_half) / n);
    }
}

// Stage twiddle table of a length-n transform with R points per thread, laid out as the
// device-side FftPlan<n, R> expects: for each stage with sub-length ns > 1 and radix rs,
// a block [r = 1..rs-1][k = 0..ns-1] of exp(-2 pi i r k / (ns rs)), computed in FP64.
template <typename T>
std::vector<twel<T>> stage_twiddles_host(int n, int R) {
    int logn = 0, logr = 0;
    while ((1 << logn) < n) ++logn;
    while ((1 << logr) < R) ++logr;
    const int nfull = logn / logr;
    const int last = 1 << (logn - nfull * logr);
    const int stages = nfull + (last > 1 ? 1 : 0);
    std::vector<twel<T>> out;
    const double two_pi = 6.283185307179586476925286766559;
    int ns = 1;
    for (int s = 0; s < stages; ++s) {
        const int rs = (s < nfull) ? R : last;
        if (ns > 1)
            for (int r = 1; r < rs; ++r)
                for (int k = 0; k < ns; ++k) {
                    const double ang = two_pi * (double)r * (double)k / ((double)ns * rs);
                    out.push_back(tw_entry<T>(std::cos(ang), -std::sin(ang)));
                }
        ns *= rs;
    }
    if (out.empty()) out.push_back(tw_entry<T>(1.0, 0.0));
    return out;
}

gpe_status dev_alloc(gpe_batch* b, void** p, size_t bytes) {
    cudaError_t e = device_malloc(p, bytes);
    if (e != cudaSuccess) {
        cudaGetLastError();
        return fail(GPE_ENOMEM, "cudaMalloc(%zu): %s", bytes, cudaGetErrorString(e));
    }
    b->allocs.push_back(*p);
    return GPE_OK;
}

// Compact form of an FP32 kinetic phase table for the x pass: (p, u) of modes 0..n/2 (the
// table is symmetric in k), possible when no entry needed a sign (every angle within
// +-pi/2, so the entry's third value is the common 1/n).  Empty otherwise.
std::vector<float2> compact_phases(const std::vector<float4>& t) {
    const int n = (int)t.size();
    std::vector<float2> c;
    for (int i = 0; i < n; ++i)
        if (!(t[i].z > 0.0f) || t[i].z != t[0].z) return c;
    for (int i = 0; i <= n / 2; ++i) c.push_back(make_float2(t[i].x, t[i].y));
    return c;
}
std::vector<float2> compact_phases(const std::vector<double2>&) { return {}; }

// FP32 stage twiddles of FftPlan<n, R> as (p, u) pairs, for kernels that take the sign of
// each rotation from its index (entry r, k of a stage with sub-length ns and radix rs is
// negative exactly when ns rs < 4 r k < 3 ns rs).  The rule is checked against every
// entry's stored sign; empty if any differs (the kernels then keep the full table).
std::vector<float2> pair_twiddles(const std::vector<float4>& t, int n, int R) {
    int logn = 0, logr = 0;
    while ((1 << logn) < n) ++logn;
    while ((1 << logr) < R) ++logr;
    const int nfull = logn / logr, last = 1 << (logn - nfull * logr), stages = nfull + (last > 1 ? 1 : 0);
    std::vector<float2> out;
    int ns = 1;
    size_t i = 0;
    for (int st = 0; st < stages; ++st) {
        const int rs = (st < nfull) ? R : last;
        if (ns > 1)
            for (int r = 1; r < rs; ++r)
                for (int k = 0; k < ns; ++k, ++i) {
                    const int64_t x4 = 4ll * r * k;
                    const bool neg = x4 > (int64_t)ns * rs && x4 < 3ll * ns * rs;
                    if (i >= t.size() || (t[i].z < 0.0f) != neg || std::fabs(t[i].z) != 1.0f) return {};
                    out.push_back(make_float2(t[i].x, t[i].y));
                }
        ns *= rs;
    }
    if (out.empty()) out.push_back(make_float2(0.0f, 0.0f));
    return out.size() == t.size() ? out : std::vector<float2>{};
}
std::vector<float2> pair_twiddles(const std::vector<double2>&, int, int) { return {}; }

template <typename T>
gpe_status build_group_tables(gpe_batch* b, Group& g) {
    for (int a = 0; a < g.ndim; ++a) {
        std::vector<twel<T>> pf, ph;
        phase_tables_host<T>(g.n[a], g.dx, b->p.dt, pf, ph);
        const size_t bytes = sizeof(twel<T>) * g.n[a];
        gpe_status s;
        if ((s = dev_alloc(b, &g.ph_full[a], bytes)) != GPE_OK) return s;
        if ((s = dev_alloc(b, &g.ph_half[a], bytes)) != GPE_OK) return s;
        GPE_CK(cudaMemcpy(g.ph_full[a], pf.data(), bytes, cudaMemcpyHostToDevice));
        GPE_CK(cudaMemcpy(g.ph_half[a], ph.data(), bytes, cudaMemcpyHostToDevice));
        if (a == 0 && g.ndim >= 2) {
            std::vector<float2> cf = compact_phases(pf), ch = compact_phases(ph);
            std::vector<float2> t2 = pair_twiddles(stage_twiddles_host<T>(g.n[0], 8), g.n[0], 8);
            // whole 16-byte units: the x pass fetches these tables with bulk copies
            for (auto* v : {&cf, &ch, &t2})
                if (!v->empty() && (v->size() & 1)) v->push_back(make_float2(0.0f, 0.0f));
            if (!cf.empty() && !ch.empty() && !t2.empty()) {
                const size_t cb = sizeof(float2) * cf.size(), tb = sizeof(float2) * t2.size();
                if ((s = dev_alloc(b, &g.phc_full, cb)) != GPE_OK) return s;
                if ((s = dev_alloc(b, &g.phc_half, cb)) != GPE_OK) return s;
                if ((s = dev_alloc(b, &g.tw2x, tb)) != GPE_OK) return s;
                GPE_CK(cudaMemcpy(g.phc_full, cf.data(), cb, cudaMemcpyHostToDevice));
                GPE_CK(cudaMemcpy(g.phc_half, ch.data(), cb, cudaMemcpyHostToDevice));
                GPE_CK(cudaMemcpy(g.tw2x, t2.data(), tb, cudaMemcpyHostToDevice));
            }
        }
        for (int ri = 0; ri < 3; ++ri) {
            const std::vector<twel<T>> tw = stage_twiddles_host<T>(g.n[a], 4 << ri);
            const size_t tb = sizeof(twel<T>) * tw.size();
            if ((s = dev_alloc(b, &g.tw[a][ri], tb)) != GPE_OK) return s;
            GPE_CK(cudaMemcpy(g.tw[a][ri], tw.data(), tb, cudaMemcpyHostToDevice));
        }
    }
    if (g.ndim == 1 && g.n[0] > resident1d_max_n<T>()) {
        const int M = res1d_cluster_block<T>();
        const int C = g.n[0] / M;
        g.cluster = C;
        gpe_status s;
        for (int ri = 0; ri < 3; ++ri) {
            const std::vector<twel<T>> tw = stage_twiddles_host<T>(M, 4 << ri);
            const size_t tb = sizeof(twel<T>) * tw.size();
            if ((s = dev_alloc(b, &g.tw_local[ri], tb)) != GPE_OK) return s;
            GPE_CK(cudaMemcpy(g.tw_local[ri], tw.data(), tb, cudaMemcpyHostToDevice));
        }
        std::vector<twel<T>> wn((size_t)C * M);
        const double two_pi = 6.283185307179586476925286766559;
        for (int r = 0; r < C; ++r)
            for (int n = 0; n < M; ++n) {
                const double ang = two_pi * (double)n * (double)r / (double)g.n[0];
                wn[(size_t)r * M + n] = tw_entry<T>(std::cos(ang), -std::sin(ang));
            }
        if ((s = dev_alloc(b, &g.wn, sizeof(twel<T>) * wn.size())) != GPE_OK) return s;
        GPE_CK(cudaMemcpy(g.wn, wn.data(), sizeof(twel<T>) * wn.size(), cudaMemcpyHostToDevice));
    }
    return GPE_OK;
}

template <typename T>
gpe_status check_sizes(const gpe_traj& t) {
    if (t.ndim == 1) {
        const int lim = 8 * res1d_cluster_block<T>();
        if (t.n[0] < 64 || t.n[0] > lim)
            return fail(GPE_EUNSUPPORTED, "1D size %d outside [64, %d]", t.n[0], lim);
    } else {
        for (int a = 0; a < t.ndim; ++a) {
            const int lim = (a == 0) ? xpass_max_n<T>() : colpass_max_n<T>();
            if (t.n[a] < 64 || t.n[a] > lim)
                return fail(GPE_EUNSUPPORTED, "axis %d size %d outside [64, %d]", a, t.n[a], lim);
        }
    }
    return GPE_OK;
}

double q_at_host(const gpe_batch* b, double t) {
    const int K = b->p.n_knots;
    if (K <= 0) return b->p.q;
    if (K == 1) return b->knots[0];
    double u = t / b->p.t_end * (double)(K - 1);
    if (u <= 0.0) return b->knots[0];
    if (u >= (double)(K - 1)) return b->knots[K - 1];
    int i = (int)std::floor(u);
    double w = u - (double)i;
    return b->knots[i] * (1.0 - w) + b->knots[i + 1] * w;
}

template <typename T>
PassArgs<T> base_args(const gpe_batch* b, const Group& g) {
    PassArgs<T> a{};
    a.ptrs = reinterpret_cast<cplx<T>* const*>(g.dptrs);
    a.comp_stride = g.sites;
    a.ntraj = g.ntraj;
    a.ncomp = 3;
    a.status = b->d_status;
    a.coef.c0 = (T)b->p.c0;
    a.coef.c1 = (T)b->p.c1;
    a.coef.dt = (T)b->p.dt;
    a.coef.q = (T)b->p.q;
    a.coef.kind = b->integrator;
    a.wait_first = b->wait_first;
    return a;
}

// Pure kinetic pass along axis ax (1 = y, 2 = z) with the full or half time step.
template <typename T>
cudaError_t col_pass(gpe_batch* b, const Group& g, int ax, bool half, cudaStream_t s) {
    ProfScope ps(b, 1, s, 1);
    if (g.contiguous) {
        const int nx = g.n[0], ny = g.n[1], nz = g.n[2];
        const int nxt = nx / g.cols[ax];
        const int n_tiles = ax == 1 ? nxt * g.ntraj * 3 * nz : nxt * ny * g.ntraj * 3;
        const twel<T>* tws[3] = {reinterpret_cast<const twel<T>*>(g.tw[ax][0]),
                                 reinterpret_cast<const twel<T>*>(g.tw[ax][1]),
                                 reinterpret_cast<const twel<T>*>(g.tw[ax][2])};
        return launch_colpass_tma<T>(g.n[ax], ax, g.cols[ax], ax == 1 ? g.map_y : g.map_z, n_tiles, nxt, ny, tws,
                                     reinterpret_cast<const twel<T>*>(half ? g.ph_half[ax] : g.ph_full[ax]),
                                     b->d_status, s, b->wait_first);
    }
    PassArgs<T> a = base_args<T>(b, g);
    for (int ri = 0; ri < 3; ++ri) a.tw[ri] = reinterpret_cast<const twel<T>*>(g.tw[ax][ri]);
    a.ph = reinterpret_cast<const twel<T>*>(half ? g.ph_half[ax] : g.ph_full[ax]);
    const int nx = g.n[0], ny = g.n[1], nz = g.n[2];
    if (ax == 1) {
        a.stride = nx;
        a.n_outer = nz;
        a.outer_stride = (int64_t)nx * ny;
    } else {
        a.stride = (int64_t)nx * ny;
        a.n_outer = ny;
        a.outer_stride = nx;
    }
    a.nx_tiles = nx / colpass_cols<T>(g.n[ax]);
    return launch_colpass<T>(g.n[ax], a, s);
}

template <typename T>
cudaError_t x_pass(gpe_batch* b, const Group& g, bool pre, bool half_post, double q, cudaStream_t s) {
    ProfScope ps(b, 0, s, 1);
    PassArgs<T> a = base_args<T>(b, g);
    for (int ri = 0; ri < 3; ++ri) a.tw[ri] = reinterpret_cast<const twel<T>*>(g.tw[0][ri]);
    a.ph_pre = reinterpret_cast<const twel<T>*>(g.ph_half[0]);
    a.ph = reinterpret_cast<const twel<T>*>(half_post ? g.ph_half[0] : g.ph_full[0]);
    if (g.phc_full) {
        a.phc = reinterpret_cast<const float2*>(half_post ? g.phc_half : g.phc_full);
        a.phc_pre = reinterpret_cast<const float2*>(g.phc_half);
        a.ph_scale = 1.0f / (float)g.n[0];
        a.tw2 = reinterpret_cast<const float2*>(g.tw2x);
    }
    a.rows_per_traj = (int64_t)g.n[1] * g.n[2];
    a.total_rows = a.rows_per_traj * g.ntraj;
    a.coef.q = (T)q;
    a.vpot = reinterpret_cast<const T*>(g.vpot);
    return launch_xpass<T>(g.n[0], pre, a, s, g.xthreads);
}

template <typename T>
gpe_status step_group(gpe_batch* b, const Group& g, int64_t nsteps, cudaStream_t s) {
    const double dt = b->p.dt;
    const double t0 = (double)b->step * dt;
    if (g.ndim == 1) {
        Res1DArgs<T> a{};
        a.ptrs = reinterpret_cast<cplx<T>* const*>(g.dptrs);
        a.ntraj = g.ntraj;
        for (int ri = 0; ri < 3; ++ri) a.tw[ri] = reinterpret_cast<const twel<T>*>(g.tw[0][ri]);
        a.ph_full = reinterpret_cast<const twel<T>*>(g.ph_full[0]);
        a.ph_half = reinterpret_cast<const twel<T>*>(g.ph_half[0]);
        a.c0 = (T)b->p.c0;
        a.c1 = (T)b->p.c1;
        a.dt = (T)dt;
        a.dt_d = dt;
        a.t0 = t0;
        a.q_const = b->p.q;
        a.t_end = b->p.t_end;
        a.knots = b->d_knots;
        a.n_knots = b->p.n_knots;
        a.nsteps = nsteps;
        a.kind = b->integrator;
        a.vpot = reinterpret_cast<const T*>(g.vpot);
        ProfScope ps(b, 2, s, 1);
        if (g.cluster > 0) {
            const twel<T>* twl = reinterpret_cast<const twel<T>*>(g.tw_local[sizeof(T) == 4 ? 2 : 1]);
            GPE_CK(launch_res1d_cluster<T>(g.n[0], a, twl, reinterpret_cast<const twel<T>*>(g.wn), s));
        } else {
            GPE_CK(launch_resident1d<T>(g.n[0], a, s));
        }
        return GPE_OK;
    }
    // K(dt/2) along the strided axes first (they commute with the x pass), then per step
    // an x pass [Kx(dt/2) on the first step] L Kx(dt or dt/2) and the strided passes.
    for (int ax = g.ndim - 1; ax >= 1; --ax) GPE_CK(col_pass<T>(b, g, ax, true, s));
    for (int64_t st = 0; st < nsteps; ++st) {
        const bool last = (st == nsteps - 1);
        const double q = q_at_host(b, t0 + ((double)st + 0.5) * dt);
        GPE_CK(x_pass<T>(b, g, st == 0, last, q, s));
        for (int ax = 1; ax < g.ndim; ++ax) GPE_CK(col_pass<T>(b, g, ax, last, s));
    }
    return GPE_OK;
}

void drop_graphs(gpe_batch* b) {
    for (auto& kv : b->graphs) cudaGraphExecDestroy(kv.second.exec);
    b->graphs.clear();
}

// Block size of the x pass that the library uses for group g when none is fixed.
int xpass_default_threads(const Group& g) {
    return (g.n[0] == 128 || g.n[0] == 1024) ? 128 : (g.n[0] == 512 ? 192 : 256);
}

// Times the x pass (no leading half kick) on nt scratch fields for each block size it is
// built for and returns the fastest (0 if nothing could be timed).
int tune_xpass_threads(gpe_batch* b, const Group& g, void* scratch, int nt, cudaEvent_t e0, cudaEvent_t e1,
                       cudaStream_t s) {
    int cand[4];
    const int nc = xpass_thread_candidates<float>(g.n[0], cand);
    if (nc == 0 || !g.phc_full) return 0;   // block sizes are built for the compact-table pass only
    void** tab = nullptr;
    if (device_malloc((void**)&tab, sizeof(void*) * nt) != cudaSuccess) {
        cudaGetLastError();
        return 0;
    }
    std::vector<void*> hp(nt);
    for (int i = 0; i < nt; ++i) hp[i] = (char*)scratch + (size_t)i * 3 * g.sites * sizeof(float2);
    int best_t = 0;
    float best = 0.f;
    if (cudaMemcpyAsync(tab, hp.data(), sizeof(void*) * nt, cudaMemcpyHostToDevice, s) == cudaSuccess) {
        PassArgs<float> a = base_args<float>(b, g);
        a.ptrs = reinterpret_cast<float2* const*>(tab);
        a.ntraj = nt;
        for (int ri = 0; ri < 3; ++ri) a.tw[ri] = reinterpret_cast<const twel<float>*>(g.tw[0][ri]);
        a.ph_pre = reinterpret_cast<const twel<float>*>(g.ph_half[0]);
        a.ph = reinterpret_cast<const twel<float>*>(g.ph_full[0]);
        if (g.phc_full) {
            a.phc = reinterpret_cast<const float2*>(g.phc_full);
            a.phc_pre = reinterpret_cast<const float2*>(g.phc_half);
            a.ph_scale = 1.0f / (float)g.n[0];
            a.tw2 = reinterpret_cast<const float2*>(g.tw2x);
        }
        a.rows_per_traj = (int64_t)g.n[1] * g.n[2];
        a.total_rows = a.rows_per_traj * nt;
        a.vpot = nullptr;
        for (int i = 0; i < nc; ++i) {
            if (launch_xpass<float>(g.n[0], false, a, s, cand[i]) != cudaSuccess) {
                cudaGetLastError();
                continue;
            }
            cudaEventRecord(e0, s);
            for (int r = 0; r < 3; ++r) launch_xpass<float>(g.n[0], false, a, s, cand[i]);
            cudaEventRecord(e1, s);
            g_launches += 4;
            float ms = 0.f;
            if (cudaEventSynchronize(e1) != cudaSuccess || cudaEventElapsedTime(&ms, e0, e1) != cudaSuccess) {
                cudaGetLastError();
                continue;
            }
            if (best == 0.f || ms < best) {
                best = ms;
                best_t = cand[i];
            }
        }
    }
    cudaStreamSynchronize(s);
    cudaFree(tab);
    return best_t;
}

// Tile autotuner.  On the first step of an FP32 batch, every 2D/3D shape group times, on a
// scratch batch shaped like its own fields -- up to 256 MiB, zero-filled: the passes' cost
// does not depend on the values -- each block size the x pass is built for and, for groups
// with back-to-back fields, each tile width the column pass is built for
// (colpass_tma_candidates), one warm-up and three timed launches per candidate on the
// caller's stream; it keeps the fastest, frees the scratch and re-encodes the group's tensor
// maps.  Neither choice changes a result bit.  Skipped while the stream is being captured
// (the defaults stay) or when disabled; sizes the caller fixed stay.
gpe_status tune_tiles(gpe_batch* b, cudaStream_t s) {
    if (!b->autotune || b->dtype != GPE_C64) return GPE_OK;
    cudaStreamCaptureStatus cs = cudaStreamCaptureStatusNone;
    if (cudaStreamIsCapturing(s, &cs) != cudaSuccess) {
        cudaGetLastError();
        return GPE_OK;
    }
    if (cs != cudaStreamCaptureStatusNone) return GPE_OK;
    for (Group& g : b->groups) {
        if (g.tuned || g.ndim < 2 || ((g.fixed || !g.contiguous) && g.xfixed)) continue;
        g.tuned = true;
        const size_t per_traj = (size_t)3 * g.sites * sizeof(float2);
        const size_t cap = ((size_t)256 << 20) / per_traj;
        const int nt = (int)std::min<size_t>((size_t)g.ntraj, cap < 1 ? 1 : cap);
        void* scratch = nullptr;
        if (device_malloc(&scratch, per_traj * nt) != cudaSuccess) {
            cudaGetLastError();
            continue;   // no room to tune: keep the defaults
        }
        cudaEvent_t e0 = nullptr, e1 = nullptr;
        bool ok = cudaMemsetAsync(scratch, 0, per_traj * nt, s) == cudaSuccess &&
                  cudaEventCreate(&e0) == cudaSuccess && cudaEventCreate(&e1) == cudaSuccess;
        if (ok && !g.xfixed) {
            const int t = tune_xpass_threads(b, g, scratch, nt, e0, e1, s);
            if (t > 0) g.xthreads = t;
        }
        const bool tune_cols = !g.fixed && g.contiguous;
        for (int ax = 1; ok && tune_cols && ax < g.ndim; ++ax) {
            int cand[8];
            const int nc = colpass_tma_candidates<float>(g.n[ax], cand);
            float best = 0.f;
            int best_c = g.cols[ax];
            const int nx = g.n[0], ny = g.n[1], nz = g.n[2];
            const twel<float>* tws[3] = {reinterpret_cast<const twel<float>*>(g.tw[ax][0]),
                                         reinterpret_cast<const twel<float>*>(g.tw[ax][1]),
                                         reinterpret_cast<const twel<float>*>(g.tw[ax][2])};
            const twel<float>* ph = reinterpret_cast<const twel<float>*>(g.ph_full[ax]);
            for (int i = 0; i < nc; ++i) {
                const int c = cand[i];
                if (nx % c) continue;
                CUtensorMap my{}, mz{};
                if (!encode_maps(&my, &mz, g, scratch, nt, 4, c, c)) continue;
                const int nxt = nx / c;
                const int n_tiles = ax == 1 ? nxt * nt * 3 * nz : nxt * ny * nt * 3;
                auto launch = [&]() {
                    return launch_colpass_tma<float>(g.n[ax], ax, c, ax == 1 ? my : mz, n_tiles, nxt, ny, tws, ph,
                                                     b->d_status, s);
                };
                if (launch() != cudaSuccess) {   // does not fit (shared memory): not a candidate here
                    cudaGetLastError();
                    continue;
                }
                cudaEventRecord(e0, s);
                for (int r = 0; r < 3; ++r) launch();
                cudaEventRecord(e1, s);
                g_launches += 4;
                float ms = 0.f;
                if (cudaEventSynchronize(e1) != cudaSuccess || cudaEventElapsedTime(&ms, e0, e1) != cudaSuccess) {
                    cudaGetLastError();
                    continue;
                }
                if (best == 0.f || ms < best) {
                    best = ms;
                    best_c = c;
                }
            }
            g.cols[ax] = best_c;
        }
        cudaStreamSynchronize(s);
        if (e0) cudaEventDestroy(e0);
        if (e1) cudaEventDestroy(e1);
        cudaFree(scratch);
        if (tune_cols && !encode_group_maps(g, 4)) return fail(GPE_ECUDA, "tensor maps after tile tuning");
    }
    return GPE_OK;
}

// Trajectory lanes of group g: how many consecutive trajectory ranges its step sequence is
// split into, each advanced on its own stream.  By default two lanes for the 2D group of a
// batch of one shape (at least two trajectories): the kernels of one lane fill the tail and
// the launch gap of the other's (measured, FP32, against one lane: 512^2 x 64 122.5 ->
// 118.6 ms per 250 steps, 1024^2 x 16 +4.6 %, 256^2 x 256 +4.4 %, 128^2 x 512 +4.3 %; four
// lanes no better).  One lane for 3D groups (256^3 x 8 3.4 % slower with two, 128^3 x 64
// 1.8 % faster), for 1D groups (one resident launch runs every step) and for every group of
// a batch of several shapes, whose groups already overlap on their own streams (the ragged
// mix of 232 trajectories in 9 groups: 143.4 ms per 250 steps with one lane per group,
// 149.8 ms with two per 2D group).  While profiling, one lane, so that each kernel is timed
// alone.  Every trajectory goes through the same kernels with the same arithmetic either
// way: the split changes no result bit.
int group_lanes(const gpe_batch* b, const Group& g) {
    if (g.ndim < 2 || b->prof.on) return 1;
    const int req = b->lanes_req >= 0 ? b->lanes_req : (g.ndim == 2 && b->groups.size() == 1 ? 2 : 1);
    return std::max(1, std::min(req, g.ntraj));
}

// Lane j of L of group g: the same tables over trajectories [t0, t0 + cnt), with the
// device pointer tables offset and, for contiguous groups, tensor maps over that range.
bool lane_view(const Group& g, int j, int L, int elem_bytes, Group& v) {
    const int t0 = (int)((int64_t)g.ntraj * j / L), t1 = (int)((int64_t)g.ntraj * (j + 1) / L);
    v = g;
    v.ntraj = t1 - t0;
    v.ids.assign(g.ids.begin() + t0, g.ids.begin() + t1);
    v.hptrs.assign(g.hptrs.begin() + t0, g.hptrs.begin() + t1);
    v.dptrs = g.dptrs + t0;
    v.d_ids = g.d_ids + t0;
    return !g.contiguous || encode_group_maps(v, elem_bytes);
}

// Streams and join events for n concurrent work items (created once, kept).
gpe_status ensure_streams(gpe_batch* b, size_t n) {
    while (b->gstream.size() < n) {
        cudaStream_t gs;
        cudaEvent_t ev;
        if (cudaStreamCreateWithFlags(&gs, cudaStreamNonBlocking) != cudaSuccess) return fail(GPE_ECUDA, "stream creation");
        b->gstream.push_back(gs);
        if (cudaEventCreateWithFlags(&ev, cudaEventDisableTiming) != cudaSuccess) return fail(GPE_ECUDA, "event creation");
        b->ev_join.push_back(ev);
    }
    return GPE_OK;
}

// All groups advance nsteps.  Each group, or each lane of it, is one work item; with
// several, each runs on its own stream, forked from and joined back into ``s``, so small
// groups overlap large ones and the lanes of a group overlap each other.
gpe_status run_steps(gpe_batch* b, int64_t nsteps, cudaStream_t s) {
    auto step = [&](const Group& g, cudaStream_t gs) {
        return (b->dtype == GPE_C64) ? step_group<float>(b, g, nsteps, gs) : step_group<double>(b, g, nsteps, gs);
    };
    size_t items = 0;
    for (const Group& g : b->groups) items += (size_t)group_lanes(b, g);
    if (items == 1) return step(b->groups[0], s);
    gpe_status st = ensure_streams(b, items);
    if (st != GPE_OK) return st;
    const int eb = b->dtype == GPE_C64 ? 4 : 8;
    GPE_CK(cudaEventRecord(b->ev_fork, s));
    size_t k = 0;
    for (const Group& g : b->groups) {
        const int L = group_lanes(b, g);
        for (int j = 0; j < L; ++j, ++k) {
            cudaStream_t gs = b->gstream[k];
            GPE_CK(cudaStreamWaitEvent(gs, b->ev_fork, 0));
            if (L == 1) {
                st = step(g, gs);
            } else {
                Group v;
                if (!lane_view(g, j, L, eb, v)) return fail(GPE_ECUDA, "tensor maps of a trajectory lane");
                st = step(v, gs);
            }
            if (st != GPE_OK) return st;
            GPE_CK(cudaEventRecord(b->ev_join[k], gs));
        }
    }
    for (size_t i = 0; i < items; ++i) GPE_CK(cudaStreamWaitEvent(s, b->ev_join[i], 0));
    return GPE_OK;
}

}  // namespace

extern "C" {

const char* gpe_last_error(void) { return g_err.c_str(); }

gpe_status gpe_batch_create(const gpe_traj* trajs, int32_t ntraj, gpe_dtype dtype, const gpe_params* params,
                            gpe_batch** out) {
    g_err.clear();
    if (!out) return fail(GPE_EINVAL, "out is NULL");
    *out = nullptr;
    if (!trajs || ntraj <= 0) return fail(GPE_EINVAL, "need ntraj > 0 trajectories");
    if (!params) return fail(GPE_EINVAL, "params is NULL");
    if (dtype != GPE_C64 && dtype != GPE_C128) return fail(GPE_EINVAL, "unknown dtype %d", (int)dtype);
    if (!(params->dt > 0.0) || !std::isfinite(params->dt)) return fail(GPE_EINVAL, "dt must be > 0");
    if (!std::isfinite(params->c0) || !std::isfinite(params->c1) || !std::isfinite(params->q))
        return fail(GPE_EINVAL, "non-finite coupling");
    if (params->n_knots < 0 || (params->n_knots > 0 && !params->q_knots))
        return fail(GPE_EINVAL, "bad q knots");
    if (params->n_knots > 1 && !(params->t_end > 0.0)) return fail(GPE_EINVAL, "t_end must be > 0 with knots");
    for (int i = 0; i < ntraj; ++i) {
        const gpe_traj& t = trajs[i];
        if (t.ndim < 1 || t.ndim > 3) return fail(GPE_EINVAL, "traj %d: ndim %d", i, t.ndim);
        for (int a = 0; a < 3; ++a) {
            if (a < t.ndim && !is_pow2(t.n[a])) return fail(GPE_EINVAL, "traj %d: n[%d]=%d not a power of two", i, a, t.n[a]);
            if (a >= t.ndim && t.n[a] != 1) return fail(GPE_EINVAL, "traj %d: unused n[%d] must be 1", i, a);
        }
        if (!(t.dx > 0.0)) return fail(GPE_EINVAL, "traj %d: dx must be > 0", i);
        if (!t.psi || ((uintptr_t)t.psi & 15u)) return fail(GPE_EINVAL, "traj %d: psi NULL or not 16-byte aligned", i);
        gpe_status s = (dtype == GPE_C64) ? check_sizes<float>(t) : check_sizes<double>(t);
        if (s != GPE_OK) return s;
    }
    gpe_batch* b = new (std::nothrow) gpe_batch();
    if (!b) return fail(GPE_ENOMEM, "host allocation failed");
    b->dtype = dtype;
    b->p = *params;
    if (params->n_knots > 0) b->knots.assign(params->q_knots, params->q_knots + params->n_knots);
    b->p.q_knots = nullptr;
    b->trajs.assign(trajs, trajs + ntraj);
    cudaGetDevice(&b->device);
    auto cleanup = [&](gpe_status s) {
        gpe_batch_destroy(b);
        return s;
    };
    gpe_status s;
    if ((s = dev_alloc(b, (void**)&b->d_status, sizeof(int))) != GPE_OK) return cleanup(s);
    if (cudaMemset(b->d_status, 0, sizeof(int)) != cudaSuccess) return cleanup(fail(GPE_ECUDA, "memset status"));
    if (!b->knots.empty()) {
        if ((s = dev_alloc(b, (void**)&b->d_knots, sizeof(double) * b->knots.size())) != GPE_OK) return cleanup(s);
        if (cudaMemcpy(b->d_knots, b->knots.data(), sizeof(double) * b->knots.size(), cudaMemcpyHostToDevice) != cudaSuccess)
            return cleanup(fail(GPE_ECUDA, "copy knots"));
    }
    // group trajectories of equal shape and spacing
    std::map<std::tuple<int, int, int, int, double>, int> gi;
    for (int i = 0; i < ntraj; ++i) {
        const gpe_traj& t = trajs[i];
        auto key = std::make_tuple(t.ndim, t.n[0], t.n[1], t.n[2], t.dx);
        auto it = gi.find(key);
        int k;
        if (it == gi.end()) {
            k = (int)b->groups.size();
            gi[key] = k;
            Group g;
            g.ndim = t.ndim;
            g.n[0] = t.n[0];
            g.n[1] = t.n[1];
            g.n[2] = t.n[2];
            g.dx = t.dx;
            g.sites = (int64_t)t.n[0] * t.n[1] * t.n[2];
            b->groups.push_back(g);
        } else {
            k = it->second;
        }
        b->groups[k].ids.push_back(i);
        b->groups[k].hptrs.push_back(t.psi);
    }
    for (Group& g : b->groups) {
        g.ntraj = (int)g.ids.size();
        if ((s = dev_alloc(b, (void**)&g.dptrs, sizeof(void*) * g.ntraj)) != GPE_OK) return cleanup(s);
        if ((s = dev_alloc(b, (void**)&g.d_ids, sizeof(int32_t) * g.ntraj)) != GPE_OK) return cleanup(s);
        if (cudaMemcpy(g.dptrs, g.hptrs.data(), sizeof(void*) * g.ntraj, cudaMemcpyHostToDevice) != cudaSuccess ||
            cudaMemcpy(g.d_ids, g.ids.data(), sizeof(int32_t) * g.ntraj, cudaMemcpyHostToDevice) != cudaSuccess)
            return cleanup(fail(GPE_ECUDA, "copy group tables"));
        s = (dtype == GPE_C64) ? build_group_tables<float>(b, g) : build_group_tables<double>(b, g);
        if (s != GPE_OK) return cleanup(s);
        const size_t vb = (dtype == GPE_C64) ? 8 : 16;
        bool contiguous = g.ndim >= 2;
        for (int i = 1; i < g.ntraj && contiguous; ++i)
            contiguous = (char*)g.hptrs[i] == (char*)g.hptrs[0] + (size_t)i * 3 * g.sites * vb;
        if (contiguous) {
            for (int ax = 1; ax < g.ndim; ++ax)
                g.cols[ax] = (dtype == GPE_C64) ? colpass_cols<float>(g.n[ax]) : colpass_cols<double>(g.n[ax]);
            contiguous = encode_group_maps(g, (int)(vb / 2));
        }
        g.contiguous = contiguous;
    }
    if (cudaStreamCreateWithFlags(&b->cap_stream, cudaStreamNonBlocking) != cudaSuccess ||
        cudaEventCreateWithFlags(&b->ev_fork, cudaEventDisableTiming) != cudaSuccess)
        return cleanup(fail(GPE_ECUDA, "stream/event creation"));
    if (b->groups.size() > 1 && (s = ensure_streams(b, b->groups.size())) != GPE_OK) return cleanup(s);
    if ((s = obs_init(b->obs, b->groups, b->dtype == GPE_C128, b->device)) != GPE_OK) {
        g_err = obs_last_error();
        return cleanup(s);
    }
    *out = b;
    return GPE_OK;
}

gpe_status gpe_batch_destroy(gpe_batch* b) {
    if (!b) return GPE_OK;
    cudaDeviceSynchronize();
    obs_free(b->obs);
    for (auto& kv : b->graphs) cudaGraphExecDestroy(kv.second.exec);
    for (cudaStream_t gs : b->gstream) cudaStreamDestroy(gs);
    for (cudaEvent_t e : b->ev_join) cudaEventDestroy(e);
    if (b->ev_fork) cudaEventDestroy(b->ev_fork);
    if (b->cap_stream) cudaStreamDestroy(b->cap_stream);
    for (cudaEvent_t e : b->prof.pool) cudaEventDestroy(e);
    for (void* p : b->allocs) cudaFree(p);
    delete b;
    return GPE_OK;
}

gpe_status tw_init_noise(gpe_batch* b, uint64_t seed, const double mean_spinor[6], double noise_per_mode,
                         void* stream) {
    g_err.clear();
    if (!b) return fail(GPE_EINVAL, "batch is NULL");
    if (!mean_spinor) return fail(GPE_EINVAL, "mean_spinor is NULL");
    if (!(noise_per_mode >= 0.0) || !std::isfinite(noise_per_mode)) return fail(GPE_EINVAL, "noise_per_mode must be >= 0");
    for (int i = 0; i < 6; ++i)
        if (!std::isfinite(mean_spinor[i])) return fail(GPE_EINVAL, "non-finite mean spinor");
    cudaStream_t s = (cudaStream_t)stream;
    if (b->traj_base + (int64_t)b->trajs.size() > 0xFFFFFFFFll) return fail(GPE_EINVAL, "trajectory index beyond 32 bits");
    for (const Group& g : b->groups) {
        NoiseArgs a{};
        a.ptrs = g.dptrs;
        a.traj_ids = g.d_ids;
        a.ntraj = g.ntraj;
        a.traj_base = (uint32_t)b->traj_base;
        a.sites = g.sites;
        a.key0 = (uint32_t)(seed & 0xFFFFFFFFu);
        a.key1 = (uint32_t)(seed >> 32);
        a.sigma = std::sqrt(noise_per_mode / std::pow(g.dx, g.ndim));
        for (int i = 0; i < 6; ++i) a.mean[i] = mean_spinor[i];
        a.mean_field = g.mean_field;
        ProfScope ps(b, 3, s, 1);
        GPE_CK(b->dtype == GPE_C64 ? launch_noise<float>(a, s) : launch_noise<double>(a, s));
    }
    b->step = 0;
    return GPE_OK;
}

gpe_status gpe_step_batch(gpe_batch* b, int64_t nsteps, void* stream) {
    g_err.clear();
    if (!b) return fail(GPE_EINVAL, "batch is NULL");
    if (nsteps < 0) return fail(GPE_EINVAL, "nsteps < 0");
    if (nsteps == 0) return GPE_OK;
    cudaStream_t s = (cudaStream_t)stream;
    {
        gpe_status ts = tune_tiles(b, s);
        if (ts != GPE_OK) return ts;
    }
    if (b->graph_mode && b->p.n_knots == 0 && !b->prof.on) {
        auto it = b->graphs.find(nsteps);
        if (it == b->graphs.end()) {
            const int64_t before = g_launches.load();
            GPE_CK(cudaStreamBeginCapture(b->cap_stream, cudaStreamCaptureModeThreadLocal));
            gpe_status st = run_steps(b, nsteps, b->cap_stream);
            cudaGraph_t graph = nullptr;
            const cudaError_t ec = cudaStreamEndCapture(b->cap_stream, &graph);
            if (st != GPE_OK) {
                if (graph) cudaGraphDestroy(graph);
                return st;
            }
            if (ec != cudaSuccess) return fail(GPE_ECUDA, "stream capture: %s", cudaGetErrorString(ec));
            cudaGraphExec_t exec = nullptr;
            const cudaError_t ei = cudaGraphInstantiate(&exec, graph, 0);
            cudaGraphDestroy(graph);
            if (ei != cudaSuccess) return fail(GPE_ECUDA, "graph instantiate: %s", cudaGetErrorString(ei));
            const int64_t n = g_launches.load() - before;
            g_launches -= n;
            it = b->graphs.emplace(nsteps, gpe_batch::GraphEntry{exec, n}).first;
        }
        GPE_CK(cudaGraphLaunch(it->second.exec, s));
        g_launches += it->second.launches;
    } else {
        gpe_status st = run_steps(b, nsteps, s);
        if (st != GPE_OK) return st;
    }
    b->step += nsteps;
    return GPE_OK;
}

gpe_status observables_accumulate(gpe_batch* b, double* acc, uint32_t flags, int32_t slot, void* stream) {
    g_err.clear();
    if (!b) return fail(GPE_EINVAL, "batch is NULL");
    if (!acc) return fail(GPE_EINVAL, "acc is NULL");
    if (slot < 0) return fail(GPE_EINVAL, "sample_slot < 0");
    if (flags & ~(GPE_OBS_SPECTRA | GPE_OBS_DIAG | GPE_OBS_WINDING)) return fail(GPE_EINVAL, "unknown flags 0x%x", flags);
    if ((flags & GPE_OBS_SPECTRA) && b->obs.nbins <= 0)
        return fail(GPE_EUNSUPPORTED, "spectra need a shape group with equal side lengths");
    const double q = q_at_host(b, (double)b->step * b->p.dt);
    ProfScope ps(b, 4, (cudaStream_t)stream, obs_launches(b->obs, b->groups, flags));
    gpe_status s = obs_accumulate(b->obs, b->groups, b->dtype == GPE_C128, b->p.c0, b->p.c1, q, acc, flags, slot,
                                  b->d_status, (cudaStream_t)stream);
    if (s != GPE_OK) g_err = obs_last_error();
    return s;
}

gpe_status gpe_obs_layout(const gpe_batch* b, int32_t* nbins, int64_t* slot_doubles) {
    if (!b || !nbins || !slot_doubles) return fail(GPE_EINVAL, "NULL argument");
    *nbins = b->obs.nbins;
    *slot_doubles = (int64_t)4 * (b->obs.nbins > 0 ? b->obs.nbins : 0) + 9 * (int64_t)b->trajs.size();
    return GPE_OK;
}

}  // extern "C"

namespace {

// Copies between a host buffer holding every trajectory of the batch in batch order, back to
// back, and the trajectories' device fields; runs of trajectories whose fields are adjacent
// on the device go as one copy.
gpe_status batch_transfer(const gpe_batch* b, void* host, bool upload, cudaStream_t s) {
    const size_t vb = b->dtype == GPE_C64 ? sizeof(float2) : sizeof(double2);
    size_t off = 0;
    for (size_t i = 0; i < b->trajs.size();) {
        char* dev = static_cast<char*>(b->trajs[i].psi);
        size_t bytes = 0, j = i;
        for (; j < b->trajs.size(); ++j) {
            const gpe_traj& t = b->trajs[j];
            if (static_cast<char*>(t.psi) != dev + bytes) break;
            bytes += vb * 3 * (size_t)t.n[0] * t.n[1] * t.n[2];
        }
        char* h = static_cast<char*>(host) + off;
        GPE_CK(upload ? cudaMemcpyAsync(dev, h, bytes, cudaMemcpyHostToDevice, s)
                      : cudaMemcpyAsync(h, dev, bytes, cudaMemcpyDeviceToHost, s));
        off += bytes;
        i = j;
    }
    return GPE_OK;
}

}  // namespace

extern "C" {

gpe_status gpe_batch_upload(gpe_batch* b, const void* host_psi, void* stream) {
    g_err.clear();
    if (!b || !host_psi) return fail(GPE_EINVAL, "NULL argument");
    return batch_transfer(b, const_cast<void*>(host_psi), true, (cudaStream_t)stream);
}

gpe_status gpe_batch_download(const gpe_batch* b, void* host_psi, void* stream) {
    g_err.clear();
    if (!b || !host_psi) return fail(GPE_EINVAL, "NULL argument");
    return batch_transfer(b, host_psi, false, (cudaStream_t)stream);
}

gpe_status gpe_obs_download(const gpe_batch* b, const double* acc, int32_t sample_slot, double* host, void* stream) {
    g_err.clear();
    if (!b || !acc || !host || sample_slot < 0) return fail(GPE_EINVAL, "NULL argument or sample_slot < 0");
    int32_t nb = 0;
    int64_t sd = 0;
    gpe_status st = gpe_obs_layout(b, &nb, &sd);
    if (st != GPE_OK) return st;
    GPE_CK(cudaMemcpyAsync(host, acc + (size_t)sample_slot * (size_t)sd, sizeof(double) * (size_t)sd,
                           cudaMemcpyDeviceToHost, (cudaStream_t)stream));
    return GPE_OK;
}

gpe_status gpe_obs_group_layout(const gpe_batch* b, int32_t traj, int32_t* nbins, int64_t* spectra_offset) {
    if (!b || !nbins || !spectra_offset || traj < 0 || traj >= (int32_t)b->trajs.size())
        return fail(GPE_EINVAL, "bad batch, trajectory or NULL argument");
    for (size_t k = 0; k < b->groups.size(); ++k)
        for (int id : b->groups[k].ids)
            if (id == traj) {
                *nbins = k < b->obs.gbins.size() ? b->obs.gbins[k].nbins : 0;
                *spectra_offset = k < b->obs.gbins.size() ? 4 * b->obs.gbins[k].offset : 0;
                return GPE_OK;
            }
    return fail(GPE_EINVAL, "trajectory %d not found", traj);
}

gpe_status gpe_bin_counts(const gpe_batch* b, int64_t* counts) {
    if (!b || !counts) return fail(GPE_EINVAL, "NULL argument");
    if (b->obs.nbins <= 0) return fail(GPE_EUNSUPPORTED, "no radial bins for this batch");
    std::memcpy(counts, b->obs.counts.data(), sizeof(int64_t) * b->obs.nbins);
    return GPE_OK;
}

int64_t gpe_batch_get_step(const gpe_batch* b) { return b ? b->step : -1; }

gpe_status gpe_batch_set_step(gpe_batch* b, int64_t step) {
    if (!b || step < 0) return fail(GPE_EINVAL, "bad batch or step");
    b->step = step;
    return GPE_OK;
}

}  // extern "C"

namespace {

template <typename T>
gpe_status adj_workspace(gpe_batch* b) {
    if (b->adj_phi) return GPE_OK;
    const Group& g = b->groups[0];
    const size_t vb = sizeof(cplx<T>);
    const int64_t nparts = std::max<int64_t>(adjoint_parts<T>(g), 152 * 8) + 16;
    gpe_status s;
    if ((s = dev_alloc(b, &b->adj_phi, vb * 3 * g.sites * g.ntraj)) != GPE_OK) return s;
    if ((s = dev_alloc(b, &b->adj_W, vb * g.sites * g.ntraj)) != GPE_OK) return s;
    if ((s = dev_alloc(b, (void**)&b->adj_ptrs, sizeof(void*) * 3 * g.ntraj)) != GPE_OK) return s;
    if ((s = dev_alloc(b, (void**)&b->adj_part, sizeof(double) * nparts)) != GPE_OK) return s;
    b->adj_nparts = nparts;
    // exp(+i dt k^2/4)/n for the strided axes: the half-step table with the rotation's
    // stored values negated (exact), so that the kinetic strided pass with it performs the
    // conjugate pass's arithmetic
    for (int ax = 1; ax < g.ndim; ++ax) {
        std::vector<twel<T>> pf, ph;
        phase_tables_host<T>(g.n[ax], g.dx, b->p.dt, pf, ph);
        for (auto& e : ph) e = conj_entry(e);
        const size_t bytes = sizeof(twel<T>) * ph.size();
        if ((s = dev_alloc(b, &b->adj_phc[ax], bytes)) != GPE_OK) return s;
        GPE_CK(cudaMemcpy(b->adj_phc[ax], ph.data(), bytes, cudaMemcpyHostToDevice));
    }
    return GPE_OK;
}

// A contiguous view of the batch's single group over the fields at ``base`` (the adjoint's
// workspace or the caller's cotangent) for the tensor-map strided passes; with ``conj`` its
// half-step tables are the conjugated ones.  False if the tensor maps cannot be encoded.
template <typename T>
bool adj_view(const gpe_batch* b, const Group& g, const void* base, bool conj, Group& v) {
    v = g;
    const size_t fb = sizeof(cplx<T>) * 3 * (size_t)g.sites;
    for (int i = 0; i < g.ntraj; ++i) v.hptrs[i] = (char*)base + i * fb;
    for (int ax = 1; ax < g.ndim; ++ax) {
        if (v.cols[ax] <= 0) v.cols[ax] = colpass_cols<T>(g.n[ax]);
        if (conj) v.ph_half[ax] = b->adj_phc[ax];
    }
    v.contiguous = encode_group_maps(v, (int)sizeof(T));
    return v.contiguous;
}

template <typename T>
PassArgs<T> adj_col_args(const gpe_batch* b, const Group& g, int ax, void** ptrs, int ncomp, bool half) {
    PassArgs<T> a{};
    a.ptrs = reinterpret_cast<cplx<T>* const*>(ptrs);
    a.comp_stride = g.sites;
    a.ntraj = g.ntraj;
    a.ncomp = ncomp;
    a.status = b->d_status;
    for (int ri = 0; ri < 3; ++ri) a.tw[ri] = reinterpret_cast<const twel<T>*>(g.tw[ax][ri]);
    a.ph = reinterpret_cast<const twel<T>*>(half ? g.ph_half[ax] : g.ph_full[ax]);
    const int nx = g.n[0], ny = g.n[1], nz = g.n[2];
    if (ax == 1) {
        a.stride = nx;
        a.n_outer = nz;
        a.outer_stride = (int64_t)nx * ny;
    } else {
        a.stride = (int64_t)nx * ny;
        a.n_outer = ny;
        a.outer_stride = nx;
    }
    a.nx_tiles = nx / colpass_cols<T>(g.n[ax]);
    return a;
}

template <typename T>
AdjArgs<T> adj_x_args(const gpe_batch* b, const Group& g, double q) {
    AdjArgs<T> a{};
    a.sites = g.sites;
    a.rows_per_traj = (int64_t)g.n[1] * g.n[2];
    a.total_rows = a.rows_per_traj * g.ntraj;
    for (int ri = 0; ri < 3; ++ri) a.tw[ri] = reinterpret_cast<const twel<T>*>(g.tw[0][ri]);
    a.ph = reinterpret_cast<const twel<T>*>(g.ph_half[0]);
    a.c0 = (T)b->p.c0;
    a.c1 = (T)b->p.c1;
    a.q = (T)q;
    a.dt = (T)b->p.dt;
    a.vpot = reinterpret_cast<const T*>(g.vpot);
    return a;
}

// Reverse step n given phi = K(dt/2) psi_n (a contiguous [ntraj][3][sites] buffer):
//   lam <- K(-dt/2) L_n^T(phi) K(-dt/2) lam,  dL/dq_n added to dLdq.
// The strided passes run as the tensor-map pass over a contiguous view of lam (the conjugate
// pass as the kinetic pass with conjugated tables), else with pointer tables.
template <typename T>
gpe_status adjoint_from_phi(gpe_batch* b, const void* phi, void* lam, int64_t step, double* dLdq, cudaStream_t s) {
    const Group& g = b->groups[0];
    const int64_t tstride = (int64_t)sizeof(cplx<T>) * 3 * g.sites;
    Group vlam;
    const bool tma = g.ndim >= 2 && adj_view<T>(b, g, lam, true, vlam);
    void** lam_ptrs = b->adj_ptrs + g.ntraj;
    if (!tma && g.ndim >= 2) {
        GPE_CK(launch_fill_ptrs(lam_ptrs, lam, tstride, g.ntraj, s));
        g_launches += 1;
    }
    auto strided = [&]() -> cudaError_t {
        for (int ax = 1; ax < g.ndim; ++ax) {
            cudaError_t e = tma ? col_pass<T>(b, vlam, ax, true, s)
                                : launch_colpass_mode<T>(g.n[ax], 2, adj_col_args<T>(b, g, ax, lam_ptrs, 3, true), s);
            if (e != cudaSuccess) return e;
        }
        return cudaSuccess;
    };
    const double t_mid = ((double)step + 0.5) * b->p.dt;
    const AdjArgs<T> xa = adj_x_args<T>(b, g, q_at_host(b, t_mid));
    g_launches += 2 * (g.ndim - 1) + 2;
    GPE_CK(strided());
    int nparts = 0;
    GPE_CK(launch_xadj<T>(g.n[0], xa, reinterpret_cast<cplx<T>*>(lam), reinterpret_cast<const cplx<T>*>(phi),
                          b->adj_part, &nparts, s));
    GPE_CK(launch_dq_final(b->adj_part, nparts, t_mid, b->p.n_knots, b->p.t_end, dLdq, s));
    GPE_CK(strided());
    return GPE_OK;
}

// phi <- K(dt/2) phi in place for a contiguous buffer (strided axes, then x).
template <typename T>
gpe_status half_kick(gpe_batch* b, void* phi, double q, cudaStream_t s) {
    const Group& g = b->groups[0];
    const int64_t tstride = (int64_t)sizeof(cplx<T>) * 3 * g.sites;
    Group v;
    if (g.ndim >= 2 && adj_view<T>(b, g, phi, false, v)) {
        for (int ax = 1; ax < g.ndim; ++ax) GPE_CK(col_pass<T>(b, v, ax, true, s));
    } else if (g.ndim >= 2) {
        void** phi_ptrs = b->adj_ptrs;
        GPE_CK(launch_fill_ptrs(phi_ptrs, phi, tstride, g.ntraj, s));
        for (int ax = 1; ax < g.ndim; ++ax)
            GPE_CK(launch_colpass_mode<T>(g.n[ax], 0, adj_col_args<T>(b, g, ax, phi_ptrs, 3, true), s));
        g_launches += 1;
    }
    GPE_CK(launch_xkin<T>(g.n[0], adj_x_args<T>(b, g, q), reinterpret_cast<cplx<T>*>(phi), false, s));
    g_launches += (g.ndim - 1) + 1;
    return GPE_OK;
}

template <typename T>
gpe_status adjoint_step_t(gpe_batch* b, const void* psi_in, void* lam, int64_t step, double* dLdq, cudaStream_t s) {
    gpe_status st = adj_workspace<T>(b);
    if (st != GPE_OK) return st;
    const Group& g = b->groups[0];
    const int64_t tstride = (int64_t)sizeof(cplx<T>) * 3 * g.sites;
    GPE_CK(cudaMemcpyAsync(b->adj_phi, psi_in, tstride * g.ntraj, cudaMemcpyDeviceToDevice, s));
    const double q = q_at_host(b, ((double)step + 0.5) * b->p.dt);
    if ((st = half_kick<T>(b, b->adj_phi, q, s)) != GPE_OK) return st;
    return adjoint_from_phi<T>(b, b->adj_phi, lam, step, dLdq, s);
}

// One checkpoint segment of 2D/3D batches: phi_{n0} = K(dt/2) psi_{n0} by a half kick of a
// copy of the checkpoint, phi_{n0+1} .. phi_{n0+nseg-1} from the batch's fields stepped with
// merged kinetic halves (after step j's strided passes the fields hold K(dt/2) psi_{n0+j+1}),
// each copied into ``states``; then the reverse sweep from those phi.
template <typename T>
gpe_status adjoint_segment_t(gpe_batch* b, const void* ckpt, void* states, int64_t n0, int64_t nseg, void* lam,
                             double* dLdq, cudaStream_t s) {
    gpe_status st = adj_workspace<T>(b);
    if (st != GPE_OK) return st;
    if ((st = tune_tiles(b, s)) != GPE_OK) return st;
    const Group& g = b->groups[0];
    const size_t fb = sizeof(cplx<T>) * 3 * (size_t)g.sites, bb = fb * (size_t)g.ntraj;
    const double dt = b->p.dt;
    GPE_CK(cudaMemcpyAsync(states, ckpt, bb, cudaMemcpyDeviceToDevice, s));
    if ((st = half_kick<T>(b, states, q_at_host(b, ((double)n0 + 0.5) * dt), s)) != GPE_OK) return st;
    if (nseg > 1) {
        const int ncopies = g.contiguous ? 1 : g.ntraj;
        const size_t cb = g.contiguous ? bb : fb;
        for (int i = 0; i < ncopies; ++i)
            GPE_CK(cudaMemcpyAsync(g.hptrs[i], (const char*)ckpt + i * fb, cb, cudaMemcpyDeviceToDevice, s));
        for (int ax = g.ndim - 1; ax >= 1; --ax) GPE_CK(col_pass<T>(b, g, ax, true, s));
        for (int64_t j = 0; j + 1 < nseg; ++j) {
            const double q = q_at_host(b, ((double)(n0 + j) + 0.5) * dt);
            GPE_CK(x_pass<T>(b, g, j == 0, false, q, s));
            for (int ax = 1; ax < g.ndim; ++ax) GPE_CK(col_pass<T>(b, g, ax, false, s));
            char* dst = (char*)states + (size_t)(j + 1) * bb;
            for (int i = 0; i < ncopies; ++i)
                GPE_CK(cudaMemcpyAsync(dst + i * fb, g.hptrs[i], cb, cudaMemcpyDeviceToDevice, s));
        }
        g_launches += (g.ndim - 1) + (nseg - 1) * g.ndim;
    }
    b->step = n0 + nseg - 1;
    for (int64_t j = nseg - 1; j >= 0; --j)
        if ((st = adjoint_from_phi<T>(b, (const char*)states + (size_t)j * bb, lam, n0 + j, dLdq, s)) != GPE_OK)
            return st;
    return GPE_OK;
}

template <typename T>
gpe_status sf_loss_t(gpe_batch* b, const void* psi, double kmin, double kmax, double* loss, void* lam_out,
                     cudaStream_t s) {
    gpe_status st = adj_workspace<T>(b);
    if (st != GPE_OK) return st;
    const Group& g = b->groups[0];
    const size_t vb = sizeof(cplx<T>);
    const int64_t total = g.sites * g.ntraj;
    cplx<T>* W = reinterpret_cast<cplx<T>*>(b->adj_W);
    void** w_ptrs = b->adj_ptrs + 2 * g.ntraj;
    GPE_CK(launch_fill_ptrs(w_ptrs, b->adj_W, (int64_t)vb * g.sites, g.ntraj, s));
    GPE_CK(launch_fperp<T>(reinterpret_cast<const cplx<T>*>(psi), W, g.sites, total, s));
    const twel<T>* twx[3] = {reinterpret_cast<const twel<T>*>(g.tw[0][0]), reinterpret_cast<const twel<T>*>(g.tw[0][1]),
                             reinterpret_cast<const twel<T>*>(g.tw[0][2])};
    const int64_t rows = (int64_t)g.ntraj * g.n[1] * g.n[2];
    GPE_CK(launch_rowfft<T>(g.n[0], W, rows, twx, s, -1));
    for (int ax = 1; ax < g.ndim; ++ax)
        GPE_CK(launch_colpass_mode<T>(g.n[ax], 1, adj_col_args<T>(b, g, ax, w_ptrs, 1, true), s));
    const double c = std::pow(g.dx, g.ndim) / ((double)g.sites * (double)g.ntraj);
    int nparts = 0;
    GPE_CK(launch_sf_mask<T>(W, g.sites, total, g.n, g.dx, kmin, kmax, c, b->adj_part, &nparts, s));
    GPE_CK(launch_sum_final(b->adj_part, nparts, loss, s));
    g_launches += 4 + (g.ndim - 1);
    if (lam_out) {
        for (int ax = 1; ax < g.ndim; ++ax)
            GPE_CK(launch_colpass_mode<T>(g.n[ax], 3, adj_col_args<T>(b, g, ax, w_ptrs, 1, true), s));
        GPE_CK(launch_rowfft<T>(g.n[0], W, rows, twx, s, +1));
        GPE_CK(launch_sf_seed<T>(reinterpret_cast<const cplx<T>*>(psi), W, reinterpret_cast<cplx<T>*>(lam_out),
                                 g.sites, total, 1.0, s));
        g_launches += 2 + (g.ndim - 1);
    }
    return GPE_OK;
}

gpe_status adj_check(const gpe_batch* b, const void* p1, const void* p2) {
    if (!b) return fail(GPE_EINVAL, "batch is NULL");
    if (b->groups.size() != 1) return fail(GPE_EUNSUPPORTED, "the adjoint needs a batch of one shape");
    if (b->groups[0].n[0] > 1024) return fail(GPE_EUNSUPPORTED, "the adjoint supports x extents up to 1024");
    if (!p1 || ((uintptr_t)p1 & 15u)) return fail(GPE_EINVAL, "field pointer NULL or not 16-byte aligned");
    if (p2 && ((uintptr_t)p2 & 15u)) return fail(GPE_EINVAL, "cotangent pointer not 16-byte aligned");
    return GPE_OK;
}

}  // namespace

extern "C" {

gpe_status gpe_adjoint_step(gpe_batch* b, const void* psi_step_in, void* lam, int64_t step_index, double* dLdq,
                            void* stream) {
    g_err.clear();
    gpe_status st = adj_check(b, psi_step_in, lam);
    if (st != GPE_OK) return st;
    if (!lam || !dLdq) return fail(GPE_EINVAL, "lam and dLdq must be non-NULL");
    if (b->integrator != GPE_INTEGRATOR_PAPER) return fail(GPE_EUNSUPPORTED, "the adjoint is written for the paper's local step");
    if (step_index < 0) return fail(GPE_EINVAL, "step_index < 0");
    cudaStream_t s = (cudaStream_t)stream;
    ProfScope ps(b, 5, s, 0);
    return b->dtype == GPE_C64 ? adjoint_step_t<float>(b, psi_step_in, lam, step_index, dLdq, s)
                               : adjoint_step_t<double>(b, psi_step_in, lam, step_index, dLdq, s);
}

gpe_status gpe_adjoint_segment(gpe_batch* b, const void* psi_ckpt, void* states, int64_t n0, int64_t nseg, void* lam,
                               double* dLdq, void* stream) {
    g_err.clear();
    gpe_status st = adj_check(b, psi_ckpt, lam);
    if (st != GPE_OK) return st;
    if (!lam || !dLdq || !states) return fail(GPE_EINVAL, "states, lam and dLdq must be non-NULL");
    if (((uintptr_t)states & 15u) != 0) return fail(GPE_EINVAL, "states not 16-byte aligned");
    if (b->integrator != GPE_INTEGRATOR_PAPER) return fail(GPE_EUNSUPPORTED, "the adjoint is written for the paper's local step");
    if (n0 < 0 || nseg < 1) return fail(GPE_EINVAL, "need n0 >= 0 and nseg >= 1");
    cudaStream_t s = (cudaStream_t)stream;
    const Group& g = b->groups[0];
    if (g.ndim >= 2) {
        ProfScope ps(b, 5, s, 0);
        return b->dtype == GPE_C64 ? adjoint_segment_t<float>(b, psi_ckpt, states, n0, nseg, lam, dLdq, s)
                                   : adjoint_segment_t<double>(b, psi_ckpt, states, n0, nseg, lam, dLdq, s);
    }
    // 1D: the resident kernel steps the batch's fields one step per call, each psi_n copied
    // out before its step, then the reverse steps from psi_n
    const size_t fb = (b->dtype == GPE_C64 ? sizeof(float2) : sizeof(double2)) * 3 * (size_t)g.sites;
    const size_t batch_bytes = fb * (size_t)g.ntraj;
    const int ncopies = g.contiguous ? 1 : g.ntraj;
    const size_t cb = g.contiguous ? batch_bytes : fb;
    for (int i = 0; i < ncopies; ++i)
        GPE_CK(cudaMemcpyAsync(g.hptrs[i], (const char*)psi_ckpt + i * fb, cb, cudaMemcpyDeviceToDevice, s));
    b->step = n0;
    for (int64_t j = 0; j < nseg; ++j) {
        char* dst = (char*)states + (size_t)j * batch_bytes;
        for (int i = 0; i < ncopies; ++i)
            GPE_CK(cudaMemcpyAsync(dst + i * fb, g.hptrs[i], cb, cudaMemcpyDeviceToDevice, s));
        if (j + 1 < nseg && (st = gpe_step_batch(b, 1, stream)) != GPE_OK) return st;
    }
    for (int64_t j = nseg - 1; j >= 0; --j) {
        st = gpe_adjoint_step(b, (const char*)states + (size_t)j * batch_bytes, lam, n0 + j, dLdq, stream);
        if (st != GPE_OK) return st;
    }
    return GPE_OK;
}

gpe_status gpe_sf_band_loss(gpe_batch* b, const void* psi, double kmin, double kmax, double* loss, void* lam_out,
                            void* stream) {
    g_err.clear();
    gpe_status st = adj_check(b, psi, lam_out);
    if (st != GPE_OK) return st;
    if (!loss) return fail(GPE_EINVAL, "loss must be non-NULL");
    if (!(kmax >= kmin)) return fail(GPE_EINVAL, "need kmin <= kmax");
    cudaStream_t s = (cudaStream_t)stream;
    return b->dtype == GPE_C64 ? sf_loss_t<float>(b, psi, kmin, kmax, loss, lam_out, s)
                               : sf_loss_t<double>(b, psi, kmin, kmax, loss, lam_out, s);
}

gpe_status gpe_profile_enable(gpe_batch* b, int32_t enable) {
    if (!b) return fail(GPE_EINVAL, "batch is NULL");
    b->prof.on = enable != 0;
    return GPE_OK;
}

gpe_status gpe_profile_read(gpe_batch* b, double* ms, int64_t* launches) {
    if (!b || !ms || !launches) return fail(GPE_EINVAL, "NULL argument");
    GPE_CK(cudaDeviceSynchronize());
    for (int k = 0; k < kProfKinds; ++k) {
        ms[k] = 0.0;
        launches[k] = 0;
    }
    for (auto& o : b->prof.open) {
        float t = 0.f;
        GPE_CK(cudaEventElapsedTime(&t, o.second.first, o.second.second));
        ms[o.first] += t;
        launches[o.first] += 1;
    }
    b->prof.open.clear();
    b->prof.used = 0;
    return GPE_OK;
}

int64_t gpe_launch_count(void) { return g_launches.load(); }

gpe_status gpe_batch_set_traj_base(gpe_batch* b, int64_t base) {
    if (!b || base < 0) return fail(GPE_EINVAL, "bad batch or base");
    b->traj_base = base;
    return GPE_OK;
}

gpe_status gpe_batch_set_integrator(gpe_batch* b, int32_t kind) {
    if (!b) return fail(GPE_EINVAL, "batch is NULL");
    if (kind != GPE_INTEGRATOR_PAPER && kind != GPE_INTEGRATOR_ROTATION) return fail(GPE_EINVAL, "unknown integrator %d", kind);
    if (kind != b->integrator) drop_graphs(b);
    b->integrator = kind;
    return GPE_OK;
}

}  // extern "C"

namespace {

// Groups whose grid is n (unused axes 1); returns how many matched.
template <typename F>
int for_shape(gpe_batch* b, const int32_t n[3], F&& f) {
    int hits = 0;
    for (Group& g : b->groups)
        if (g.n[0] == n[0] && g.n[1] == n[1] && g.n[2] == n[2]) {
            f(g);
            ++hits;
        }
    return hits;
}

}  // namespace

extern "C" {

gpe_status gpe_batch_set_potential(gpe_batch* b, const int32_t n[3], const void* V) {
    g_err.clear();
    if (!b || !n) return fail(GPE_EINVAL, "batch or n is NULL");
    const size_t eb = b->dtype == GPE_C64 ? sizeof(float) : sizeof(double);
    if (V && ((uintptr_t)V % eb)) return fail(GPE_EINVAL, "potential not aligned to its element size");
    if (for_shape(b, n, [&](Group& g) { g.vpot = V; }) == 0)
        return fail(GPE_EINVAL, "no trajectories of shape %d x %d x %d", n[0], n[1], n[2]);
    drop_graphs(b);
    return GPE_OK;
}

gpe_status gpe_batch_set_mean_field(gpe_batch* b, const int32_t n[3], const double* mean_field) {
    g_err.clear();
    if (!b || !n) return fail(GPE_EINVAL, "batch or n is NULL");
    if (mean_field && ((uintptr_t)mean_field % 16)) return fail(GPE_EINVAL, "mean field not 16-byte aligned");
    if (for_shape(b, n, [&](Group& g) { g.mean_field = mean_field; }) == 0)
        return fail(GPE_EINVAL, "no trajectories of shape %d x %d x %d", n[0], n[1], n[2]);
    return GPE_OK;
}

gpe_status gpe_batch_set_autotune(gpe_batch* b, int32_t enable) {
    if (!b) return fail(GPE_EINVAL, "batch is NULL");
    b->autotune = enable != 0;
    return GPE_OK;
}

gpe_status gpe_batch_set_tiles(gpe_batch* b, int32_t traj, int32_t cols_y, int32_t cols_z) {
    g_err.clear();
    if (!b || traj < 0 || traj >= (int32_t)b->trajs.size()) return fail(GPE_EINVAL, "bad batch or trajectory");
    Group* gp = nullptr;
    for (Group& g : b->groups)
        for (int id : g.ids)
            if (id == traj) gp = &g;
    if (!gp) return fail(GPE_EINVAL, "trajectory %d not found", traj);
    Group& g = *gp;
    if (b->dtype != GPE_C64 || !g.contiguous || g.ndim < 2)
        return fail(GPE_EUNSUPPORTED, "tile widths are selectable for FP32 2D/3D groups with back-to-back fields");
    if (cols_y < 0 || cols_z < 0 || (g.ndim < 3 && cols_z != 0)) return fail(GPE_EINVAL, "bad tile widths");
    const int want[3] = {0, cols_y, cols_z};
    for (int ax = 1; ax < g.ndim; ++ax) {
        if (want[ax] == 0) continue;
        int cand[8];
        const int nc = colpass_tma_candidates<float>(g.n[ax], cand);
        bool built = false;
        for (int i = 0; i < nc; ++i) built = built || cand[i] == want[ax];
        if (!built || g.n[0] % want[ax])
            return fail(GPE_EINVAL, "tile width %d is not built for n = %d (nx = %d)", want[ax], g.n[ax], g.n[0]);
    }
    for (int ax = 1; ax < g.ndim; ++ax)
        if (want[ax]) g.cols[ax] = want[ax];
    g.fixed = true;
    if (!encode_group_maps(g, 4)) return fail(GPE_ECUDA, "tensor maps for the new tile widths");
    drop_graphs(b);
    return GPE_OK;
}

gpe_status gpe_batch_set_xpass_threads(gpe_batch* b, int32_t traj, int32_t threads) {
    g_err.clear();
    if (!b || traj < 0 || traj >= (int32_t)b->trajs.size()) return fail(GPE_EINVAL, "bad batch or trajectory");
    Group* gp = nullptr;
    for (Group& g : b->groups)
        for (int id : g.ids)
            if (id == traj) gp = &g;
    if (!gp) return fail(GPE_EINVAL, "trajectory %d not found", traj);
    if (b->dtype != GPE_C64 || gp->ndim < 2 || !gp->phc_full)
        return fail(GPE_EUNSUPPORTED,
                    "the x-pass block size is selectable for FP32 2D/3D groups whose kinetic angles are within "
                    "pi/2 (dt < dx^2 / pi)");
    int cand[4];
    const int nc = xpass_thread_candidates<float>(gp->n[0], cand);
    bool built = threads == 0;
    for (int i = 0; i < nc; ++i) built = built || cand[i] == threads;
    if (!built) return fail(GPE_EINVAL, "x-pass block size %d is not built", threads);
    gp->xthreads = threads;
    gp->xfixed = true;
    drop_graphs(b);
    return GPE_OK;
}

gpe_status gpe_batch_get_xpass_threads(const gpe_batch* b, int32_t traj, int32_t* threads) {
    if (!b || !threads || traj < 0 || traj >= (int32_t)b->trajs.size()) return fail(GPE_EINVAL, "bad batch or trajectory");
    for (const Group& g : b->groups)
        for (int id : g.ids)
            if (id == traj) {
                *threads = g.ndim < 2 ? 0 : (g.xthreads > 0 ? g.xthreads : xpass_default_threads(g));
                return GPE_OK;
            }
    return fail(GPE_EINVAL, "trajectory %d not found", traj);
}

gpe_status gpe_batch_get_tiles(const gpe_batch* b, int32_t traj, int32_t cols[2], int32_t* tuned) {
    if (!b || !cols || traj < 0 || traj >= (int32_t)b->trajs.size()) return fail(GPE_EINVAL, "bad batch or trajectory");
    for (const Group& g : b->groups)
        for (int id : g.ids)
            if (id == traj) {
                cols[0] = g.contiguous ? g.cols[1] : 0;
                cols[1] = g.contiguous && g.ndim == 3 ? g.cols[2] : 0;
                if (tuned) *tuned = g.tuned ? 1 : 0;
                return GPE_OK;
            }
    return fail(GPE_EINVAL, "trajectory %d not found", traj);
}

gpe_status gpe_batch_set_wait_limit(gpe_batch* b, int64_t first_wait_polls) {
    g_err.clear();
    if (!b) return fail(GPE_EINVAL, "batch is NULL");
    if (first_wait_polls < -1 || first_wait_polls >= (int64_t)0xFFFFFFFFu)
        return fail(GPE_EINVAL, "first_wait_polls must be -1 (default) or in [0, 2^32 - 1)");
    b->wait_first = first_wait_polls < 0 ? 0u : (uint32_t)(first_wait_polls + 1);
    drop_graphs(b);
    return GPE_OK;
}

gpe_status gpe_debug_fail_alloc(int64_t after) {
    g_alloc_fail_after.store(after < 0 ? -1 : after);
    return GPE_OK;
}

gpe_status gpe_debug_table_memory(int32_t mode) {
    g_err.clear();
    if (mode != 0 && mode != 1) return fail(GPE_EINVAL, "table memory mode must be 0 or 1");
    g_table_tmem.store(mode);
    return GPE_OK;
}

gpe_status gpe_batch_set_graph(gpe_batch* b, int32_t enable) {
    if (!b) return fail(GPE_EINVAL, "batch is NULL");
    b->graph_mode = enable != 0;
    return GPE_OK;
}

gpe_status gpe_batch_set_lanes(gpe_batch* b, int32_t lanes) {
    g_err.clear();
    if (!b) return fail(GPE_EINVAL, "batch is NULL");
    if (lanes != -1 && (lanes < 1 || lanes > 64)) return fail(GPE_EINVAL, "lanes must be -1 or 1..64");
    if (lanes != b->lanes_req) drop_graphs(b);
    b->lanes_req = lanes;
    return GPE_OK;
}

gpe_status gpe_batch_get_lanes(const gpe_batch* b, int32_t traj, int32_t* lanes) {
    g_err.clear();
    if (!b || !lanes) return fail(GPE_EINVAL, "NULL argument");
    if (traj < 0 || traj >= (int32_t)b->trajs.size()) return fail(GPE_EINVAL, "trajectory index out of range");
    for (const Group& g : b->groups)
        for (int id : g.ids)
            if (id == traj) {
                *lanes = group_lanes(b, g);
                return GPE_OK;
            }
    return fail(GPE_EINVAL, "trajectory not in any group");
}

}  // extern "C"

namespace {

// Checkpoint file: "GPECKPT1", version, the batch's configuration (dtype, integrator,
// step, trajectory base, couplings, q knots, every trajectory's shape and spacing), the
// fields of every trajectory, and an FNV-1a hash of all preceding bytes.
constexpr char kCkptMagic[8] = {'G', 'P', 'E', 'C', 'K', 'P', 'T', '1'};
constexpr uint32_t kCkptVersion = 1;

uint64_t fnv1a(const unsigned char* p, size_t n) {
    uint64_t h = 1469598103934665603ull;
    for (size_t i = 0; i < n; ++i) {
        h ^= p[i];
        h *= 1099511628211ull;
    }
    return h;
}

struct Writer {
    std::vector<unsigned char> buf;
    template <typename X> void put(const X& x) {
        const unsigned char* p = reinterpret_cast<const unsigned char*>(&x);
        buf.insert(buf.end(), p, p + sizeof(X));
    }
};

struct Reader {
    const std::vector<unsigned char>& buf;
    size_t pos = 0;
    template <typename X> bool get(X& x) {
        if (pos + sizeof(X) > buf.size()) return false;
        std::memcpy(&x, buf.data() + pos, sizeof(X));
        pos += sizeof(X);
        return true;
    }
};

size_t field_bytes(const gpe_batch* b, const gpe_traj& t) {
    return (size_t)3 * t.n[0] * t.n[1] * t.n[2] * (b->dtype == GPE_C64 ? 8 : 16);
}

void put_config(Writer& w, const gpe_batch* b) {
    w.put((int32_t)b->dtype);
    w.put((int32_t)b->trajs.size());
    w.put((int32_t)b->integrator);
    w.put(b->p.c0);
    w.put(b->p.c1);
    w.put(b->p.q);
    w.put(b->p.dt);
    w.put(b->p.t_end);
    w.put((int32_t)b->knots.size());
    for (double k : b->knots) w.put(k);
    for (const gpe_traj& t : b->trajs) {
        w.put(t.ndim);
        for (int a = 0; a < 3; ++a) w.put(t.n[a]);
        w.put(t.dx);
    }
}

}  // namespace

extern "C" {

gpe_status gpe_batch_save(const gpe_batch* b, const char* path, void* stream) {
    g_err.clear();
    if (!b || !path) return fail(GPE_EINVAL, "batch or path is NULL");
    GPE_CK(cudaStreamSynchronize((cudaStream_t)stream));
    Writer w;
    for (char c : kCkptMagic) w.put(c);
    w.put(kCkptVersion);
    w.put(b->step);
    w.put(b->traj_base);
    put_config(w, b);
    for (const gpe_traj& t : b->trajs) {
        const size_t nb = field_bytes(b, t);
        const size_t at = w.buf.size();
        try {
            w.buf.resize(at + nb);
        } catch (const std::bad_alloc&) {
            return fail(GPE_ENOMEM, "host buffer of %zu bytes", at + nb);
        }
        GPE_CK(cudaMemcpy(w.buf.data() + at, t.psi, nb, cudaMemcpyDeviceToHost));
    }
    w.put(fnv1a(w.buf.data(), w.buf.size()));
    FILE* f = std::fopen(path, "wb");
    if (!f) return fail(GPE_EINVAL, "cannot open %s for writing", path);
    const size_t wrote = std::fwrite(w.buf.data(), 1, w.buf.size(), f);
    const int closed = std::fclose(f);
    if (wrote != w.buf.size() || closed != 0) return fail(GPE_EINVAL, "short write to %s", path);
    return GPE_OK;
}

gpe_status gpe_batch_load(gpe_batch* b, const char* path, void* stream) {
    g_err.clear();
    if (!b || !path) return fail(GPE_EINVAL, "batch or path is NULL");
    FILE* f = std::fopen(path, "rb");
    if (!f) return fail(GPE_EINVAL, "cannot open %s", path);
    std::vector<unsigned char> buf;
    {
        unsigned char chunk[1 << 16];
        size_t n;
        while ((n = std::fread(chunk, 1, sizeof(chunk), f)) > 0) buf.insert(buf.end(), chunk, chunk + n);
        std::fclose(f);
    }
    if (buf.size() < sizeof(kCkptMagic) + sizeof(uint64_t) ||
        std::memcmp(buf.data(), kCkptMagic, sizeof(kCkptMagic)) != 0)
        return fail(GPE_EINVAL, "%s is not a checkpoint of this library", path);
    uint64_t h = 0;
    std::memcpy(&h, buf.data() + buf.size() - sizeof(uint64_t), sizeof(uint64_t));
    if (fnv1a(buf.data(), buf.size() - sizeof(uint64_t)) != h) return fail(GPE_EINVAL, "%s is corrupt (hash)", path);
    Reader r{buf};
    r.pos = sizeof(kCkptMagic);
    uint32_t version = 0;
    int64_t step = 0, base = 0;
    if (!r.get(version) || version != kCkptVersion) return fail(GPE_EINVAL, "checkpoint version %u", version);
    if (!r.get(step) || !r.get(base)) return fail(GPE_EINVAL, "truncated checkpoint");
    // the configuration must be the batch's own, byte for byte
    Writer mine;
    put_config(mine, b);
    if (r.pos + mine.buf.size() > buf.size() ||
        std::memcmp(buf.data() + r.pos, mine.buf.data(), mine.buf.size()) != 0)
        return fail(GPE_EINVAL, "checkpoint of another batch configuration (dtype, integrator, couplings, q knots, "
                                "shapes or spacing differ)");
    r.pos += mine.buf.size();
    size_t need = 0;
    for (const gpe_traj& t : b->trajs) need += field_bytes(b, t);
    if (r.pos + need + sizeof(uint64_t) != buf.size()) return fail(GPE_EINVAL, "checkpoint size does not match the batch");
    GPE_CK(cudaStreamSynchronize((cudaStream_t)stream));
    for (const gpe_traj& t : b->trajs) {
        const size_t nb = field_bytes(b, t);
        GPE_CK(cudaMemcpy(t.psi, buf.data() + r.pos, nb, cudaMemcpyHostToDevice));
        r.pos += nb;
    }
    b->step = step;
    b->traj_base = base;
    return GPE_OK;
}

gpe_status gpe_sync_status(gpe_batch* b, void* stream) {
    g_err.clear();
    if (!b) return fail(GPE_EINVAL, "batch is NULL");
    GPE_CK(cudaStreamSynchronize((cudaStream_t)stream));
    int st = 0;
    GPE_CK(cudaMemcpy(&st, b->d_status, sizeof(int), cudaMemcpyDeviceToHost));
    GPE_CK(cudaMemset(b->d_status, 0, sizeof(int)));
    if (st != 0) return fail((gpe_status)st, "device status %d", st);
    return GPE_OK;
}

}  // extern "C"
