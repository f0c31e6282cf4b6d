// Host runtime and C ABI of the photometric bundle adjustment library: the
// context, input validation, point reordering into tiles, the (tile, frame)
// entry lists, the workspace layout, uploads, and the IC / FC iteration
// drivers that enqueue the kernels on the caller's stream.
#include <algorithm>
#include <cmath>
#include <cstdarg>
#include <cstdio>
#include <cstring>
#include <map>
#include <new>
#include <string>
#include <thread>
#include <atomic>
#include <condition_variable>
#include <functional>
#include <mutex>
#include <tuple>
#include <vector>

#include "pba_chol.cuh"
#include "pba_kernels.cuh"
#include "pba_mlp.cuh"

using namespace pba;

namespace {

constexpr size_t kAlign = 256;

size_t align_up(size_t x) { return (x + kAlign - 1) & ~(kAlign - 1); }

uint32_t spread16(uint32_t x)
{
    x &= 0xffffu;
    x = (x | (x << 8)) & 0x00ff00ffu;
    x = (x | (x << 4)) & 0x0f0f0f0fu;
    x = (x | (x << 2)) & 0x33333333u;
    x = (x | (x << 1)) & 0x55555555u;
    return x;
}

// Host parallelism of the structure build: a fixed set of worker threads
// (up to 15 beside the caller, created on first use and kept for the
// process), so that a build over many small bundles does not pay a thread
// start per range. run(k, fn) calls fn(i) for every i < k, the caller
// taking part, and returns when all have returned; one run at a time.
class HostPool {
  public:
    static HostPool& get()
    {
        static HostPool pool;
        return pool;
    }
    int threads() const { return (int)workers_.size() + 1; }

    void run(int k, const std::function<void(int)>& fn)
    {
        if (k <= 1 || workers_.empty()) {
            for (int i = 0; i < k; ++i) fn(i);
            return;
        }
        std::lock_guard<std::mutex> one(run_m_);
        uint64_t g;
        {
            std::lock_guard<std::mutex> lk(m_);
            g = ++gen_;
            job_ = &fn;
            k_ = k;
            left_ = k;
            next_.store((g & 0xffffffffu) << 32);  // this run's generation, index 0
        }
        cv_.notify_all();
        work(g, &fn, k);
        std::unique_lock<std::mutex> lk(m_);
        done_cv_.wait(lk, [this]() { return left_ == 0; });
        job_ = nullptr;
    }

    ~HostPool()
    {
        {
            std::lock_guard<std::mutex> lk(m_);
            stop_ = true;
            ++gen_;
        }
        cv_.notify_all();
        for (std::thread& t : workers_) t.join();
    }

  private:
    HostPool()
    {
        const int hw = std::max(1, std::min(16, (int)std::thread::hardware_concurrency()));
        for (int i = 1; i < hw; ++i) workers_.emplace_back([this]() { loop(); });
    }
    // Takes indices of run g until none is left. An index is taken by
    // advancing the counter only while it still holds run g's generation,
    // so a thread that arrives late never takes a later run's index.
    void work(uint64_t g, const std::function<void(int)>* job, int k)
    {
        const uint64_t tag = (g & 0xffffffffu) << 32;
        for (;;) {
            uint64_t v = next_.load();
            for (;;) {
                if ((v & ~0xffffffffull) != tag || (int)(v & 0xffffffffu) >= k) return;
                if (next_.compare_exchange_weak(v, v + 1)) break;
            }
            (*job)((int)(v & 0xffffffffu));
            std::lock_guard<std::mutex> lk(m_);
            if (--left_ == 0) done_cv_.notify_one();
        }
    }
    void loop()
    {
        uint64_t seen = 0;
        for (;;) {
            uint64_t g;
            const std::function<void(int)>* job;
            int k;
            {
                std::unique_lock<std::mutex> lk(m_);
                cv_.wait(lk, [&]() { return gen_ != seen; });
                seen = g = gen_;
                if (stop_) return;
                job = job_;
                k = k_;
            }
            if (job) work(g, job, k);
        }
    }
    std::vector<std::thread> workers_;
    std::mutex m_, run_m_;
    std::condition_variable cv_, done_cv_;
    const std::function<void(int)>* job_ = nullptr;
    int k_ = 0, left_ = 0;
    std::atomic<uint64_t> next_{0};
    uint64_t gen_ = 0;
    bool stop_ = false;
};

// The number of contiguous ranges of at least `grain` of n items the
// structure build splits a loop into (at most max_parts and the pool's
// threads).
int parallel_parts(int64_t n, int64_t grain, int max_parts = 16)
{
    return (int)std::max<int64_t>(1, std::min<int64_t>({(int64_t)HostPool::get().threads(), (int64_t)max_parts,
                                                        n / std::max<int64_t>(1, grain)}));
}

// fn(k, begin, end) for the parallel_parts(n, grain, max_parts) ranges
// (range k = [n k / parts, n (k + 1) / parts)), on the pool's threads
template <class Fn>
void parallel_ranges(int64_t n, int64_t grain, int max_parts, Fn&& fn)
{
    const int k = parallel_parts(n, grain, max_parts);
    if (k == 1) {
        fn(0, (int64_t)0, n);
        return;
    }
    HostPool::get().run(k, [&](int i) { fn(i, n * i / k, n * (i + 1) / k); });
}

// Timing slots (pba_last_timing): precompute, residual pass, reduce,
// Schur/assemble, factor/solve/update, final evaluation, per-point kernels.
enum { TS_PRE = 0, TS_PASS, TS_REDUCE, TS_SCHUR, TS_SOLVE, TS_EVAL, TS_POINT, TS_N };
static_assert(TS_N == PBA_TIMING_SLOTS, "timing slots");

using TimedPair = std::pair<int, std::pair<cudaEvent_t, cudaEvent_t>>;

// A captured launch sequence: replaying it submits every kernel of a call
// with one cudaGraphLaunch (the host no longer paces the small kernels).
struct GraphRec {
    cudaGraphExec_t exec = nullptr;
    std::vector<TimedPair> tev;  // event pairs recorded by the graph's nodes
    int64_t launches = 0;        // kernels per replay
};

// graph key: (kind, iterations, timing mask)
enum { G_ITERATE = 0, G_FC = 1, G_PRECOMPUTE = 2, G_SOLVE = 3 };
using GraphKey = std::tuple<int, int, int>;  // (kind, iterations [+ re-anchoring period << 16], timing)

}  // namespace

// Inputs of one bundle as the caller gave them, and its place in the
// concatenated problem.
struct BundleIn {
    bool have_frames = false, have_points = false;
    int F = 0;
    const void* images = nullptr;
    std::vector<double> poses_init;  // F*12
    int N = 0;
    std::vector<int32_t> uv;
    std::vector<double> d_init;
    // set by pba_set_points from the caller's visibility (which is not
    // kept): the bundle's tiles of 32 points in Morton order and its
    // (tile, frame) entries, frames in order within a tile
    int F_pts = 0;                    // frame count the entries were formed for
    int T = 0;
    std::vector<int> perm;            // slot (within the bundle's tiles) -> caller index, -1 for pads
    std::vector<int> tile_ent;        // T + 1 offsets of each tile's local entries
    std::vector<int> ent_f;           // local frame of each local entry
    std::vector<unsigned> ent_mask;   // lanes (points of the tile) the entry's frame sees
    // set by build_structure
    int fo = 0, to = 0, e0 = 0, e1 = 0;
    int64_t V = 0;
    int64_t item0 = 0;  // the bundle's first Schur pair item
};

struct pba_ctx {
    pba_config cfg{};
    std::vector<int32_t> pattern;
    cudaStream_t stream = nullptr;
    std::string err = "no error";

    // bundles (cfg.n_bundles); they share the camera: image size, pitch,
    // element type, memory kind and intrinsics
    int B = 1;
    std::vector<BundleIn> bun;
    int W = 0, H = 0, pitch = 0;
    pba_dtype dtype = PBA_F32;
    pba_memory mem = PBA_MEM_DEVICE;
    double K[4] = {0, 0, 0, 0};

    // derived host structures over all bundles (frames, tiles, entries and
    // frame pairs concatenated bundle after bundle)
    bool built = false;
    int F = 0, N = 0;  // total frames and points
    int T = 0, Npad = 0, E = 0, NC = 0, Fmax = 0, n6max = 0;
    int64_t V = 0;
    std::vector<Entry> entries;
    std::vector<int> tile_entry, frame_entry, entry_slot, frame_bundle, tile_f0;
    std::vector<BundleDesc> bdesc;
    int64_t n_so = 0, n_ao = 0, n_lo = 0;  // sizes of the per-bundle system arrays
    int n_po = 0, n_cmap = 0;
    std::vector<int> pair_fg, pair_chunk, chunk_pair, chunk_start;  // sparse Schur lists
    std::vector<int2> pair_items;  // placed only for the SIMT path (fill_pair_items)
    int64_t n_pair_items = 0;
    bool items_ready = false;
    // tensor-core Schur complement: super-tiles (first row, frames, first
    // tile, tiles), their frame rows and the output blocks
    std::vector<int4> st_info, st_items;
    std::vector<StRow> st_rows;
    int schur_path = PBA_SCHUR_AUTO;
    int n_sm = 0;  // SMs of the context's device (the automatic Schur path choice)
    bool ic_chunks_valid = false;  // ic_schur_part holds every chunk of the last IC formation

    // workspace
    bool ws_ready = false, ic_ready = false;
    char* ws = nullptr;
    size_t ws_bytes = 0;
    struct {
        void* img;
        float *gx, *gy;
        int* pat;
        Entry* entries;
        int *tile_entry, *frame_entry, *entry_slot, *frame_bundle, *tile_f0, *slot_caller;
        float *ic_part, *ic_hpart;  // per-entry IC H_ff sums and J_d^T W_0 J_d (kept for window updates)
        unsigned char* todo;        // F: frames whose entries a window update must precompute
        unsigned char* tile_todo;   // T: tiles that see a frame that entered or left the window
        BundleDesc* bund;
        int* uvs;
        float2* xn;
        float* I0p;
        unsigned char* valid_pt;
        double *d64, *d0_64, *dd_last, *inv_hnn, *inv_d0;
        float *gn_ic, *Hnn_ic, *gn_fc, *Hnn_fc;
        float4* J4;
        float *Hfd_ic, *Hfd_fc;
        float* ent_part;
        TileStats* tstats;
        float *fc, *fc_prev, *dthsq;
        float2* dth2;
        float *dcur, *dprev, *gpart, *ddsq_t;
        float2* G0p;
        float4* estats;
        double *poses64, *poses0_64, *dtheta64;
        double *red_ic, *red_y, *red_photo;
        double *Soff, *S_ic, *S_fc;
        dfloat* Sinv2;  // IC S^-1 over the active frames (double-float, compact)
        dfloat *A2, *L2, *Linv, *dpiv, *rpiv;  // double-float factorisation (IC and FC in turn)
        int *pair_fg, *pair_chunk, *chunk_pair, *chunk_start;
        int2* pair_items;
        float2* schur_part;     // FC: chunk sums of the Schur complement (every iteration)
        float2* ic_schur_part;  // IC: chunk sums at p_0, kept for window updates
        int4 *st_info, *st_items;
        StRow* st_rows;
        short *st_ea, *st_eb;
        long long* schur_acc;   // fixed-point S_off sums of the tensor-core path (zero between formations)
        // joint brightness unknowns (cfg.photometric = 2, one bundle): the
        // per-pair H_a and p_0 masks, the H_pa / H_aa frame sums, the border
        // sums of S, and the 8 (F - 1) system's factorisation and inverse
        float* Had;
        unsigned* vmask0;
        double* red_aff;
        float* Had_fc;     // FC: per pair J_d^T W [-v, -1]
        float* aff_part;   // FC: E rows of kEntryPartial (the 15 H_pa / H_aa sums)
        double* red_aff_fc;
        long long* aff_acc;
        dfloat *A8, *L8, *Linv8, *dpiv8, *rpiv8, *Sinv8;
        double* dab64;
        float2* dab2;
        int *active_ic, *active_fc, *cmap_ic, *cmap_fc;
        int* err;
        double* stats;
    } d{};
    int stats_slots = 0;
    int last_fc = 0;  // which system the last update came from
    int ldl_cluster = 0;  // CTAs per bundle of the factorisation (0: default)
    std::vector<int> bundle_err;  // per-bundle error bits of the last check
    // sliding window: frames outside it keep their data but their entries
    // are uploaded with no visible lane, so no kernel sees their residuals
    std::vector<unsigned char> frame_on, frame_todo;  // F
    // F: frames that entered or left since the last IC (pre)computation; the
    // Schur terms of every point they see change
    std::vector<unsigned char> frame_changed;
    bool window_dirty = false;  // the window changed after the last (pre)computation
    int res_warps = 8;    // warps per CTA of the IC residual pass
    bool tuned = false;

    // instrumentation
    int timing = 0;  // slot mask
    int64_t h2d = 0, d2h = 0;
    int64_t launches = 0;
    double tms[TS_N] = {};
    int64_t tcount[TS_N] = {};
    std::vector<TimedPair> tev;        // pooled events recorded by direct launches
    std::vector<TimedPair> tev_graph;  // events of replayed graphs (owned by the graphs)
    std::vector<cudaEvent_t> evpool;

    // captured launch sequences (cfg.use_graphs with a non-null stream)
    bool capturing = false;
    std::map<GraphKey, GraphRec> graphs;
};

namespace {

pba_status fail(pba_ctx* c, pba_status s, const char* fmt, ...)
{
    char buf[512];
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(buf, sizeof buf, fmt, ap);
    va_end(ap);
    c->err = buf;
    return s;
}

#define CK(call)                                                                              \
    do {                                                                                      \
        cudaError_t e_ = (call);                                                              \
        if (e_ != cudaSuccess)                                                                \
            return fail(ctx, PBA_ERR_CUDA, "%s failed: %s", #call, cudaGetErrorString(e_)); \
    } while (0)

#define LAUNCH(slot, call)            \
    do {                              \
        int ev_ = tbegin(ctx, slot);  \
        CK(call);                     \
        ++ctx->launches;              \
        tend(ctx, ev_);               \
    } while (0)

#define CHECK_BUNDLE()                                                                         \
    do {                                                                                       \
        if (!ctx) return PBA_ERR_ARG;                                                          \
        if (bundle < 0 || bundle >= ctx->B)                                                    \
            return fail(ctx, PBA_ERR_ARG, "bundle %d out of range (%d bundles)", bundle, ctx->B); \
    } while (0)

// for launchers that enqueue several kernels and count them in `nl`
#define LAUNCHN(slot, call)           \
    do {                              \
        int ev_ = tbegin(ctx, slot);  \
        int nl = 0;                   \
        CK(call);                     \
        ctx->launches += nl;          \
        tend(ctx, ev_);               \
    } while (0)

cudaEvent_t take_event(pba_ctx* ctx)
{
    if (!ctx->evpool.empty()) {
        cudaEvent_t e = ctx->evpool.back();
        ctx->evpool.pop_back();
        return e;
    }
    cudaEvent_t e = nullptr;
    cudaEventCreate(&e);
    return e;
}

int tbegin(pba_ctx* ctx, int slot)
{
    if (!((ctx->timing >> slot) & 1)) return -1;
    cudaEvent_t a = take_event(ctx), b = take_event(ctx);
    // inside a capture the pair becomes event-record nodes of the graph
    if (ctx->capturing) cudaEventRecordWithFlags(a, ctx->stream, cudaEventRecordExternal);
    else cudaEventRecord(a, ctx->stream);
    ctx->tev.push_back({slot, {a, b}});
    return (int)ctx->tev.size() - 1;
}

void tend(pba_ctx* ctx, int idx)
{
    if (idx < 0) return;
    if (ctx->capturing) cudaEventRecordWithFlags(ctx->tev[idx].second.second, ctx->stream, cudaEventRecordExternal);
    else cudaEventRecord(ctx->tev[idx].second.second, ctx->stream);
}

void tcollect(pba_ctx* ctx)
{
    for (auto& ev : ctx->tev) {
        float ms = 0.0f;
        if (cudaEventElapsedTime(&ms, ev.second.first, ev.second.second) == cudaSuccess) {
            ctx->tms[ev.first] += ms;
            ctx->tcount[ev.first] += 1;
        }
        ctx->evpool.push_back(ev.second.first);
        ctx->evpool.push_back(ev.second.second);
    }
    ctx->tev.clear();
    for (auto& ev : ctx->tev_graph) {
        float ms = 0.0f;
        if (cudaEventElapsedTime(&ms, ev.second.first, ev.second.second) == cudaSuccess) {
            ctx->tms[ev.first] += ms;
            ctx->tcount[ev.first] += 1;
        }
    }
    ctx->tev_graph.clear();
}

void destroy_graphs(pba_ctx* ctx)
{
    if (ctx->graphs.empty()) return;
    cudaStreamSynchronize(ctx->stream);
    tcollect(ctx);
    for (auto& kv : ctx->graphs) {
        if (kv.second.exec) cudaGraphExecDestroy(kv.second.exec);
        for (auto& ev : kv.second.tev) {
            ctx->evpool.push_back(ev.second.first);
            ctx->evpool.push_back(ev.second.second);
        }
    }
    ctx->graphs.clear();
}

size_t elem_size(pba_dtype t) { return t == PBA_F32 ? 4 : 2; }

cudaError_t h2d(pba_ctx* ctx, void* dst, const void* src, size_t bytes)
{
    ctx->h2d += (int64_t)bytes;
    return cudaMemcpyAsync(dst, src, bytes, cudaMemcpyHostToDevice, ctx->stream);
}

cudaError_t d2h(pba_ctx* ctx, void* dst, const void* src, size_t bytes)
{
    ctx->d2h += (int64_t)bytes;
    cudaError_t e = cudaMemcpyAsync(dst, src, bytes, cudaMemcpyDeviceToHost, ctx->stream);
    return e == cudaSuccess ? cudaStreamSynchronize(ctx->stream) : e;
}

// The context keeps its own copy of the image stack (in the workspace) when
// the images come from the host, or when several bundles' stacks must be
// made one contiguous array.
bool own_images(const pba_ctx* c) { return c->mem == PBA_MEM_HOST || c->B > 1; }

// The affine brightness pairs as unknowns of the IC system (cfg.photometric = 2).
bool joint_brightness(const pba_ctx* c) { return c->cfg.photometric == 2; }

// Lays out (and optionally assigns) the workspace; returns its size.
size_t layout(pba_ctx* c, char* base)
{
    size_t off = 0;
    auto take = [&](auto*& ptr, size_t bytes) {
        using P = std::remove_reference_t<decltype(ptr)>;
        ptr = base ? reinterpret_cast<P>(base + off) : nullptr;
        off += align_up(std::max<size_t>(bytes, 1));
    };
    const size_t F = c->F, HW = (size_t)c->H * c->W, Np = c->Npad;
    if (own_images(c)) {
        void*& img = c->d.img;
        char* p = nullptr;
        take(p, F * c->H * c->pitch * elem_size(c->dtype));
        if (base) img = p;
    }
    take(c->d.gx, F * HW * 4);
    take(c->d.gy, F * HW * 4);
    take(c->d.pat, c->pattern.size() * sizeof(int));
    take(c->d.entries, (size_t)c->E * sizeof(Entry));
    take(c->d.tile_entry, (size_t)(c->T + 1) * 4);
    take(c->d.frame_entry, (F + 1) * 4);
    take(c->d.entry_slot, (size_t)c->E * 4);
    take(c->d.frame_bundle, F * 4);
    take(c->d.tile_f0, (size_t)c->T * 4);
    take(c->d.bund, (size_t)c->B * sizeof(BundleDesc));
    take(c->d.slot_caller, Np * 4);
    take(c->d.uvs, Np * 8);
    take(c->d.xn, Np * 8);
    take(c->d.I0p, (size_t)c->T * (c->pattern.size() / 2) * kTile * 4);
    take(c->d.valid_pt, Np);
    take(c->d.d64, Np * 8);
    take(c->d.d0_64, Np * 8);
    take(c->d.dd_last, Np * 8);
    take(c->d.inv_hnn, Np * 8);
    take(c->d.inv_d0, Np * 8);
    take(c->d.gn_ic, Np * 4);
    take(c->d.Hnn_ic, Np * 4);
    take(c->d.gn_fc, Np * 4);
    take(c->d.Hnn_fc, Np * 4);
    take(c->d.J4, (size_t)c->V * c->NC * 16);
    take(c->d.Hfd_ic, (size_t)c->V * 6 * 4);
    take(c->d.Hfd_fc, (size_t)c->V * 6 * 4);
    take(c->d.ent_part, (size_t)c->E * kEntryPartial * 4);
    take(c->d.ic_part, (size_t)c->E * kEntryPartial * 4);
    take(c->d.ic_hpart, (size_t)c->E * kTile * 4);
    take(c->d.todo, F);
    take(c->d.tile_todo, (size_t)c->T);
    take(c->d.tstats, (size_t)c->T * sizeof(TileStats));
    take(c->d.fc, F * kFrameConst * 4);
    take(c->d.fc_prev, F * 12 * 4);
    take(c->d.dth2, F * 6 * sizeof(float2));
    take(c->d.dcur, Np * 4);
    take(c->d.dprev, Np * 4);
    take(c->d.gpart, (size_t)c->E * kTile * 2 * 4);  // FC: g and H_dd per (entry, lane)
    take(c->d.estats, (size_t)c->E * sizeof(float4));
    take(c->d.ddsq_t, (size_t)c->T * 4);
    take(c->d.G0p, (size_t)c->T * (c->pattern.size() / 2) * kTile * sizeof(float2));
    take(c->d.dthsq, F * 4);
    take(c->d.poses64, F * 12 * 8);
    take(c->d.poses0_64, F * 12 * 8);
    take(c->d.dtheta64, F * 6 * 8);
    take(c->d.red_ic, F * 21 * 8);
    take(c->d.red_y, F * 27 * 8);
    take(c->d.red_photo, F * 5 * 8);
    take(c->d.Soff, (size_t)c->n_so * 8);
    take(c->d.S_ic, (size_t)c->n_so * 8);
    take(c->d.Sinv2, (size_t)c->n_so * sizeof(dfloat));
    take(c->d.S_fc, (size_t)c->n_so * 8);
    take(c->d.A2, (size_t)c->n_ao * sizeof(dfloat));
    take(c->d.L2, (size_t)c->n_ao * sizeof(dfloat));
    take(c->d.Linv, (size_t)c->n_lo * sizeof(dfloat));
    take(c->d.dpiv, (size_t)c->n_po * sizeof(dfloat));
    take(c->d.rpiv, (size_t)c->n_po * sizeof(dfloat));
    take(c->d.pair_fg, c->pair_fg.size() * sizeof(int));
    take(c->d.pair_chunk, c->pair_chunk.size() * sizeof(int));
    take(c->d.chunk_pair, c->chunk_pair.size() * sizeof(int));
    take(c->d.chunk_start, c->chunk_start.size() * sizeof(int));
    take(c->d.pair_items, (size_t)c->n_pair_items * sizeof(int2));
    take(c->d.schur_part, c->chunk_pair.size() * 36 * sizeof(float2));
    take(c->d.ic_schur_part, c->chunk_pair.size() * 36 * sizeof(float2));
    take(c->d.st_info, c->st_info.size() * sizeof(int4));
    take(c->d.st_items, c->st_items.size() * sizeof(int4));
    take(c->d.st_rows, c->st_rows.size() * sizeof(StRow));
    take(c->d.st_ea, c->st_rows.size() * 6 * sizeof(short));
    take(c->d.st_eb, c->st_rows.size() * 6 * sizeof(short));
    take(c->d.schur_acc, (size_t)c->n_so * sizeof(long long));
    {
        // joint brightness unknowns (zero-sized otherwise)
        const bool jb = joint_brightness(c);
        const size_t n8 = jb ? 8 * (F - 1) : 0, n2 = jb ? 2 * (F - 1) : 0, n6 = jb ? 6 * (F - 1) : 0;
        take(c->d.Had, jb ? (size_t)c->V * 2 * 4 : 0);
        take(c->d.vmask0, jb ? (size_t)c->V * 4 : 0);
        take(c->d.red_aff, jb ? F * kAffComp * 8 : 0);
        take(c->d.Had_fc, jb ? (size_t)c->V * 2 * 4 : 0);
        take(c->d.aff_part, jb ? (size_t)c->E * kEntryPartial * 4 : 0);
        take(c->d.red_aff_fc, jb ? F * kAffComp * 8 : 0);
        take(c->d.aff_acc, (n6 * n2 + n2 * n2) * sizeof(long long));
        take(c->d.A8, (n8 + 1) * n8 * sizeof(dfloat));
        take(c->d.L8, (n8 + 1) * n8 * sizeof(dfloat));
        take(c->d.Linv8, (n8 + kLdlBlock - 1) / kLdlBlock * kLinvStride * sizeof(dfloat));
        take(c->d.dpiv8, n8 * sizeof(dfloat));
        take(c->d.rpiv8, n8 * sizeof(dfloat));
        take(c->d.Sinv8, n8 * n8 * sizeof(dfloat));
        take(c->d.dab64, jb ? F * 2 * 8 : 0);
        take(c->d.dab2, jb ? F * 2 * sizeof(float2) : 0);
    }
    take(c->d.active_ic, F * 4);
    take(c->d.active_fc, F * 4);
    take(c->d.cmap_ic, (size_t)c->n_cmap * 4);
    take(c->d.cmap_fc, (size_t)c->n_cmap * 4);
    take(c->d.err, (size_t)(1 + c->B) * 4);
    take(c->d.stats, (size_t)(c->stats_slots) * kStats * 8);
    return off;
}

bool all_set(const pba_ctx* c)
{
    for (const BundleIn& b : c->bun)
        if (!b.have_frames || !b.have_points) return false;
    return true;
}

// Sorted point order, tiles, (tile, frame) entries, frame pairs and the
// per-bundle system offsets, bundle after bundle (frames, tiles and entries
// of bundle b follow those of bundle b - 1).
// The bundle's tiles (32 points in Morton order of their pixels, ties in
// caller order) and its (tile, frame) entries, frames in order within a
// tile, from the caller's visibility (N x F bytes, null: every point in
// every frame; frame 0 is the reference and is no entry's frame). Each
// point's visibility row is read once.
void form_tiles(BundleIn& b, const uint8_t* vis)
{
    const int N = b.N, F = b.F;
    // a stable LSD radix sort of the 32-bit codes, eight bits per pass;
    // each pass counts the digits of contiguous ranges of keys in parallel
    // and places each range's keys at its offsets (digit-major, then range
    // order: stable)
    std::vector<uint64_t> key(N), tmp(N);  // code in the high half, caller index in the low
    parallel_ranges(N, 4096, 16, [&](int, int64_t i0, int64_t i1) {
        for (int64_t n = i0; n < i1; ++n) {
            const uint32_t u = (uint32_t)b.uv[2 * n], v = (uint32_t)b.uv[2 * n + 1];
            key[n] = ((uint64_t)(spread16(u) | (spread16(v) << 1)) << 32) | (uint32_t)n;
        }
    });
    const int parts = parallel_parts(N, 4096);
    std::vector<int64_t> hist((size_t)parts * 256);
    for (int shift = 32; shift < 64; shift += 8) {
        std::fill(hist.begin(), hist.end(), 0);
        parallel_ranges(N, 4096, 16, [&](int k, int64_t i0, int64_t i1) {
            int64_t* h = hist.data() + (size_t)k * 256;
            for (int64_t i = i0; i < i1; ++i) ++h[(key[i] >> shift) & 255u];
        });
        int64_t o = 0;
        for (int d = 0; d < 256; ++d)
            for (int k = 0; k < parts; ++k) {
                const int64_t c = hist[(size_t)k * 256 + d];
                hist[(size_t)k * 256 + d] = o;
                o += c;
            }
        parallel_ranges(N, 4096, 16, [&](int k, int64_t i0, int64_t i1) {
            int64_t* h = hist.data() + (size_t)k * 256;
            for (int64_t i = i0; i < i1; ++i) tmp[h[(key[i] >> shift) & 255u]++] = key[i];
        });
        key.swap(tmp);
    }
    const int T = (N + kTile - 1) / kTile;
    b.T = T;
    b.F_pts = F;
    b.perm.assign((size_t)T * kTile, -1);
    for (int i = 0; i < N; ++i) b.perm[i] = (int)(uint32_t)key[i];
    // each tile's frame masks, then the entries (the frames with a nonzero
    // mask) at the tile's offset
    std::vector<unsigned> masks((size_t)T * F);
    std::vector<int> cnt((size_t)T + 1, 0);
    parallel_ranges(T, 64, 16, [&](int, int64_t t0, int64_t t1) {
        for (int64_t t = t0; t < t1; ++t) {
            unsigned* __restrict__ mk = masks.data() + (size_t)t * F;
            std::fill(mk, mk + F, 0u);
            for (int l = 0; l < kTile; ++l) {
                const int n = b.perm[t * kTile + l];
                if (n < 0) continue;
                const unsigned bit = 1u << l;
                if (!vis) {
                    for (int f = 1; f < F; ++f) mk[f] |= bit;
                    continue;
                }
                const uint8_t* __restrict__ vr = vis + (size_t)n * F;
                for (int f = 1; f < F; ++f) mk[f] |= (unsigned)(vr[f] != 0) * bit;
            }
            int c = 0;
            for (int f = 1; f < F; ++f) c += mk[f] != 0u;
            cnt[t + 1] = c;
        }
    });
    for (int t = 0; t < T; ++t) cnt[t + 1] += cnt[t];
    b.ent_f.resize(cnt[T]);
    b.ent_mask.resize(cnt[T]);
    parallel_ranges(T, 64, 16, [&](int, int64_t t0, int64_t t1) {
        for (int64_t t = t0; t < t1; ++t) {
            const unsigned* mk = masks.data() + (size_t)t * F;
            int o = cnt[t];
            for (int f = 1; f < F; ++f)
                if (mk[f]) {
                    b.ent_f[o] = f;
                    b.ent_mask[o] = mk[f];
                    ++o;
                }
        }
    });
    b.tile_ent.swap(cnt);
}

// The (entry, entry) items of bundle b's tiles per frame pair f <= g: cnt
// (resized to npairs + 1) receives the prefix sums of the counts per pair
// (pair index of (f, g) = first pair of f + g - f), and with items non-null
// every item is placed at items[cnt[pair] + its rank in tile order] as
// (global entry of f, global entry of g). A counting sort over contiguous
// tile ranges, one host thread each, the ranges' counts placed in range
// order, so the order is the serial one.
void bundle_pair_items(const pba_ctx* c, const BundleIn& b, std::vector<int64_t>& cnt, int2* items)
{
    const int F = b.F;
    const std::vector<int>& tile_ent0 = b.tile_ent;
    std::vector<int64_t> pbase((size_t)F + 1, 0);
    for (int f = 1; f < F; ++f) pbase[f + 1] = pbase[f] + (F - f);
    const int64_t npairs = pbase[F];
    auto tile_items = [&](int64_t t, auto&& fn) {
        for (int i = tile_ent0[t]; i < tile_ent0[t + 1]; ++i) {
            const Entry& A = c->entries[b.e0 + i];
            const int fa = A.f - b.fo;
            for (int j = i; j < tile_ent0[t + 1]; ++j) {
                const Entry& Bj = c->entries[b.e0 + j];
                if (!(A.mask & Bj.mask)) continue;
                fn(pbase[fa] + (Bj.f - b.fo - fa), b.e0 + i, b.e0 + j);
            }
        }
    };
    const int max_parts =
        (int)std::max<int64_t>(1, std::min<int64_t>(16, (int64_t)(1 << 22) / std::max<int64_t>(1, npairs)));
    const int parts = parallel_parts(b.T, 64, max_parts);
    std::vector<int64_t> pc((size_t)parts * npairs, 0);  // per range: items per pair
    parallel_ranges(b.T, 64, max_parts, [&](int k, int64_t t0, int64_t t1) {
        int64_t* ck = pc.data() + (size_t)k * npairs;
        for (int64_t t = t0; t < t1; ++t) tile_items(t, [&](int64_t pid, int, int) { ++ck[pid]; });
    });
    cnt.assign((size_t)npairs + 1, 0);
    for (int64_t q = 0; q < npairs; ++q) {
        int64_t o = cnt[q];
        for (int k = 0; k < parts; ++k) {
            const int64_t n_k = pc[(size_t)k * npairs + q];
            pc[(size_t)k * npairs + q] = o;  // the range's first slot of the pair
            o += n_k;
        }
        cnt[q + 1] = o;
    }
    if (!items) return;
    parallel_ranges(b.T, 64, max_parts, [&](int k, int64_t t0, int64_t t1) {
        int64_t* put = pc.data() + (size_t)k * npairs;
        for (int64_t t = t0; t < t1; ++t)
            tile_items(t, [&](int64_t pid, int ea, int eb) { items[put[pid]++] = make_int2(ea, eb); });
    });
}

void build_structure(pba_ctx* c)
{
    c->F = c->N = c->T = 0;
    c->V = 0;
    c->Fmax = c->n6max = 0;
    c->entries.clear();
    c->tile_entry.clear();
    c->frame_bundle.clear();
    c->tile_f0.clear();
    c->bdesc.clear();
    c->n_so = c->n_ao = c->n_lo = 0;
    c->n_po = c->n_cmap = 0;
    c->pair_fg.clear();
    c->pair_chunk.assign(1, 0);
    c->chunk_pair.clear();
    c->chunk_start.assign(1, 0);
    c->pair_items.clear();
    c->n_pair_items = 0;
    c->items_ready = false;
    c->st_info.clear();
    c->st_items.clear();
    c->st_rows.clear();
    c->NC = (7 * (int)(c->pattern.size() / 2) + 3) / 4;
    int64_t pairs = 0;
    {
        size_t total = 0;
        for (const BundleIn& b : c->bun) total += b.ent_f.size();
        c->entries.reserve(total);
    }
    for (int bi = 0; bi < c->B; ++bi) {
        BundleIn& b = c->bun[bi];
        const int N = b.N, F = b.F;
        b.fo = c->F;
        b.to = c->T;
        b.e0 = (int)c->entries.size();
        // the bundle's entries (formed by pba_set_points) at the global
        // frame, tile and pair offsets
        const std::vector<int>& tile_ent0 = b.tile_ent;  // the tile's first entry (local)
        const int64_t pairs0 = pairs;
        for (int t = 0; t < b.T; ++t) {
            c->tile_entry.push_back((int)c->entries.size());
            c->tile_f0.push_back(b.fo);
            for (int i = tile_ent0[t]; i < tile_ent0[t + 1]; ++i) {
                c->entries.push_back(Entry{b.fo + b.ent_f[i], b.ent_mask[i], (int)pairs, b.to + t});
                pairs += __builtin_popcount(b.ent_mask[i]);
            }
        }
        b.e1 = (int)c->entries.size();
        b.V = pairs - pairs0;
        // frame pairs f <= g of the bundle with the (entry, entry) items of
        // the tiles that see both, in tile order (the sparse Schur kernel's
        // fixed summation order), cut into chunks of at most kSchurChunk
        // items: counted here, placed by fill_pair_items when the SIMT path
        // is in use (the tensor-core path does not read them)
        std::vector<int64_t> pbase((size_t)F + 1, 0);  // first pair index of frame f
        for (int f = 1; f < F; ++f) pbase[f + 1] = pbase[f] + (F - f);
        std::vector<int64_t> cnt;
        bundle_pair_items(c, b, cnt, nullptr);
        const size_t item0 = (size_t)c->n_pair_items;
        b.item0 = c->n_pair_items;
        c->n_pair_items += cnt.back();
        for (int f = 1; f < F; ++f)
            for (int g = f; g < F; ++g) {
                const int p = (int)c->pair_fg.size() / 2;
                const int64_t pid = pbase[f] + (g - f);
                for (int64_t i0 = cnt[pid]; i0 < cnt[pid + 1]; i0 += kSchurChunk) {
                    c->chunk_pair.push_back(p);
                    c->chunk_start.push_back((int)(item0 + std::min(i0 + kSchurChunk, cnt[pid + 1])));
                }
                c->pair_fg.push_back(b.fo + f);
                c->pair_fg.push_back(b.fo + g);
                c->pair_chunk.push_back((int)c->chunk_pair.size());
            }
        // super-tiles of kStTiles consecutive tiles for the tensor-core Schur
        // complement: the frames any of their tiles sees, in frame order,
        // with each tile's entry of the frame, and the output blocks (128
        // rows x 80 columns of the super-tile's 6-per-frame rows) that reach
        // the upper block triangle
        {
            std::vector<int> frow(F, -1);
            for (int t0 = 0; t0 < b.T; t0 += kStTiles) {
                const int nt = std::min(kStTiles, b.T - t0);
                const int row0 = (int)c->st_rows.size();
                for (int j = 0; j < nt; ++j)
                    for (int i = tile_ent0[t0 + j]; i < tile_ent0[t0 + j + 1]; ++i)
                        frow[c->entries[b.e0 + i].f - b.fo] = 0;
                for (int f = 1; f < F; ++f)
                    if (frow[f] == 0) {
                        frow[f] = (int)c->st_rows.size() - row0;
                        c->st_rows.push_back(StRow{b.fo + f, {-1, -1, -1, -1}});
                    }
                for (int j = 0; j < nt; ++j)
                    for (int i = tile_ent0[t0 + j]; i < tile_ent0[t0 + j + 1]; ++i) {
                        const int f = c->entries[b.e0 + i].f - b.fo;
                        c->st_rows[row0 + frow[f]].e[j] = b.e0 + i;
                    }
                const int nfr = (int)c->st_rows.size() - row0;
                for (int f = 1; f < F; ++f) frow[f] = -1;
                if (nfr == 0) continue;
                const int sidx = (int)c->st_info.size();
                c->st_info.push_back(make_int4(row0, nfr, b.to + t0, nt));
                const int nr = 6 * nfr;
                for (int mt = 0; mt * kSchurTcM < nr; ++mt)
                    for (int nb = 0; nb * kSchurTcN < nr; ++nb)
                        if ((mt * kSchurTcM) / 6 <= (std::min(nr, (nb + 1) * kSchurTcN) - 1) / 6)
                            c->st_items.push_back(make_int4(sidx, mt, nb, 0));
            }
        }
        const int64_t n6 = 6 * (F - 1);
        BundleDesc bd{};
        bd.fo = b.fo;
        bd.F = F;
        bd.co = c->n_cmap;
        bd.po = c->n_po;
        bd.so = c->n_so;
        bd.ao = c->n_ao;
        bd.lo = c->n_lo;
        c->bdesc.push_back(bd);
        c->n_so += n6 * n6;
        c->n_ao += (n6 + 1) * n6;
        c->n_lo += (n6 + kLdlBlock - 1) / kLdlBlock * kLinvStride;
        c->n_po += (int)n6;
        c->n_cmap += F + 1;
        for (int f = 0; f < F; ++f) c->frame_bundle.push_back(bi);
        c->F += F;
        c->N += N;
        c->T += b.T;
        c->Fmax = std::max(c->Fmax, F);
        c->n6max = std::max(c->n6max, (int)n6);
    }
    c->tile_entry.push_back((int)c->entries.size());
    c->Npad = c->T * kTile;
    c->E = (int)c->entries.size();
    c->V = pairs;
    const int F = c->F;
    c->frame_entry.assign(F + 1, 0);
    for (const Entry& e : c->entries) c->frame_entry[e.f + 1]++;
    for (int f = 0; f < F; ++f) c->frame_entry[f + 1] += c->frame_entry[f];
    // partial sums of entry e go to row entry_slot[e]: frame-major, tile
    // order within a frame (the reduction's fixed order, contiguous per frame)
    c->entry_slot.assign(c->E, 0);
    std::vector<int> fill(c->frame_entry.begin(), c->frame_entry.end() - 1);
    for (int e = 0; e < c->E; ++e) c->entry_slot[e] = fill[c->entries[e].f]++;
    c->built = true;
}

// Builds the concatenated structure once every bundle has frames and points.
pba_status ensure_structure(pba_ctx* ctx)
{
    if (!all_set(ctx)) return fail(ctx, PBA_ERR_STATE, "frames and points of every bundle must be set first");
    if (ctx->built) return PBA_OK;
    int64_t frames = 0;
    for (const BundleIn& b : ctx->bun) frames += b.F;
    if ((double)frames * ctx->H * ctx->pitch >= 4294967296.0)
        return fail(ctx, PBA_ERR_ARG, "image stack too large (frames * h * pitch over all bundles must stay below 2^32)");
    build_structure(ctx);
    if (ctx->V >= 2147483647LL)
        return fail(ctx, PBA_ERR_ARG, "too many (point, frame) observations (limit 2^31 - 1)");
    return PBA_OK;
}

SolveArgs make_solve(pba_ctx* c);

// Uploads the parameters of bundle b (poses F_b*12, depths in the caller's
// point order, nullable); the FP32 pass constants are formed on the device.
pba_status upload_params(pba_ctx* ctx, int bi, const double* poses, const double* depth, int init_photo = 0)
{
    const BundleIn& b = ctx->bun[bi];
    CK(h2d(ctx, ctx->d.poses64 + (size_t)12 * b.fo, poses, sizeof(double) * 12 * b.F));
    CK(launch_frame_consts(make_solve(ctx), b.fo, b.F, ctx->stream, init_photo));
    if (depth) {
        std::vector<double> ds(b.perm.size());
        parallel_ranges((int64_t)ds.size(), 8192, 16, [&](int, int64_t i0, int64_t i1) {
            for (int64_t i = i0; i < i1; ++i) ds[i] = b.perm[i] >= 0 ? depth[b.perm[i]] : 1.0;
        });
        CK(h2d(ctx, ctx->d.d64 + (size_t)kTile * b.to, ds.data(), sizeof(double) * ds.size()));
    }
    // all host staging above is pageable: the copies have consumed it on return
    CK(cudaStreamSynchronize(ctx->stream));
    return PBA_OK;
}

// Reads the device error words: the context's and, when it is set, every
// bundle's (kept for pba_bundle_errors), then clears them.
pba_status check_device_error(pba_ctx* ctx)
{
    int herr = 0;
    CK(d2h(ctx, &herr, ctx->d.err, sizeof(int)));
    tcollect(ctx);
    ctx->bundle_err.assign(ctx->B, 0);
    if (!herr) return PBA_OK;
    CK(d2h(ctx, ctx->bundle_err.data(), ctx->d.err + 1, sizeof(int) * ctx->B));
    CK(cudaMemsetAsync(ctx->d.err, 0, sizeof(int) * (1 + ctx->B), ctx->stream));
    std::string which;
    int nbad = 0;
    for (int b = 0; b < ctx->B; ++b)
        if (ctx->bundle_err[b]) {
            if (nbad < 8) which += (nbad ? ", " : "") + std::to_string(b);
            ++nbad;
        }
    if (nbad > 8) which += ", ...";
    const std::string where = ctx->B > 1 ? " (bundle" + std::string(nbad > 1 ? "s " : " ") + which + ")" : "";
    if (herr & kErrNotPD)
        return fail(ctx, PBA_ERR_NOT_PD, "reduced camera system is not positive definite%s", where.c_str());
    if (herr & kErrTimeout) return fail(ctx, PBA_ERR_TIMEOUT, "a tensor-core wait gave up");
    return fail(ctx, PBA_ERR_NONFINITE, "non-finite update%s", where.c_str());
}

LaunchCtx make_launch(pba_ctx* c)
{
    LaunchCtx L{};
    DevProblem& pb = L.pb;
    pb.F = c->F;
    pb.N = c->N;
    pb.Npad = c->Npad;
    pb.T = c->T;
    pb.E = c->E;
    pb.P = (int)c->pattern.size() / 2;
    pb.W = c->W;
    pb.H = c->H;
    pb.pitch = c->pitch;
    pb.dtype = c->dtype;
    pb.fx = (float)c->K[0];
    pb.fy = (float)c->K[1];
    pb.cx = (float)c->K[2];
    pb.cy = (float)c->K[3];
    pb.huber_k = (float)c->cfg.huber_k;
    pb.damp1 = (float)(1.0 + c->cfg.damping);
    pb.img = own_images(c) ? c->d.img : c->bun[0].images;
    pb.gx = c->d.gx;
    pb.gy = c->d.gy;
    pb.pat = c->d.pat;
    pb.entries = c->d.entries;
    pb.tile_entry = c->d.tile_entry;
    pb.frame_entry = c->d.frame_entry;
    pb.entry_slot = c->d.entry_slot;
    pb.frame_bundle = c->d.frame_bundle;
    pb.bund = c->d.bund;
    pb.tile_f0 = c->d.tile_f0;
    pb.uvs = c->d.uvs;
    pb.xn = c->d.xn;
    pb.I0p = c->d.I0p;
    pb.valid_pt = c->d.valid_pt;
    L.fs = FrameState{c->d.fc, c->d.fc_prev, c->d.dth2, c->d.dtheta64};
    L.it = IterBufs{c->d.dcur, c->d.dprev, c->d.gpart, c->d.estats, c->d.ddsq_t, c->d.G0p};
    L.ds_ic = DepthState{c->d.d64, c->d.d0_64, c->d.gn_ic, c->d.Hnn_ic, c->d.Hfd_ic, nullptr, c->d.dd_last,
                         c->d.err};
    L.ds_fc = DepthState{c->d.d64, c->d.d0_64, c->d.gn_fc, c->d.Hnn_fc, c->d.Hfd_fc, nullptr, c->d.dd_last,
                         c->d.err};
    L.ic = IcStore{c->d.J4, c->d.Hfd_ic, c->d.Hnn_ic, c->d.inv_hnn, c->d.inv_d0, c->d.ic_part, c->d.ic_hpart,
                   nullptr, nullptr};
    L.Hfd_fc = c->d.Hfd_fc;
    L.ent_part = c->d.ent_part;
    L.tstats = c->d.tstats;
    L.dthsq = c->d.dthsq;
    L.stats = c->d.stats;
    L.poses0 = c->d.poses0_64;
    L.stream = c->stream;
    L.res_warps = c->res_warps;
    L.photo = c->cfg.photometric;
    if (joint_brightness(c)) {
        L.ic.Had = c->d.Had;
        L.ic.vmask0 = c->d.vmask0;
        L.ds_ic.Had = c->d.Had;
        L.pb.vmask0 = c->d.vmask0;
        L.pb.Had = c->d.Had;
        L.Had_fc = c->d.Had_fc;
        L.aff_part = c->d.aff_part;
        L.ds_fc.Had = c->d.Had_fc;
    }
    return L;
}

SchurLists schur_lists(pba_ctx* c)
{
    return SchurLists{c->d.pair_fg, c->d.pair_chunk, c->d.chunk_pair, c->d.chunk_start,
                      c->d.pair_items, (int)c->pair_fg.size() / 2, (int)c->chunk_pair.size()};
}

// The automatic choice: the tensor cores once the bundle set has at least
// four output blocks of the tensor-core formation per SM (below that the
// SIMT former's co-visible items are fewer than the tensor path's fixed
// per-block work: helix30, 30 frames, 20,000 points, forms S in 23 us on
// the SIMT pipes against 40 us; orbit101 in 1.17 ms on the tensor cores
// against 1.91 ms)
int effective_schur_path(const pba_ctx* c)
{
    if (c->schur_path != PBA_SCHUR_AUTO) return c->schur_path;
    return (int64_t)c->st_items.size() >= 4 * (int64_t)(c->n_sm > 0 ? c->n_sm : 152) ? PBA_SCHUR_TENSOR
                                                                                    : PBA_SCHUR_SIMT;
}

SchurTcLists schur_tc_lists(pba_ctx* c)
{
    return SchurTcLists{c->d.st_info, c->d.st_rows, c->d.st_items, c->d.st_ea, c->d.st_eb, c->d.schur_acc,
                        (int)c->st_info.size(), (int)c->st_items.size()};
}

// S_off from the H_fd and H_dd of a system (red: its frame sums, H_ff
// first) by the selected path; part / tile_todo: the SIMT path's chunk sums
// and, for a window update, the tiles whose chunks are formed again
cudaError_t launch_schur(pba_ctx* c, const DevProblem& pb, const float* Hfd, const float* Hnn, const double* red,
                         int red_stride, float2* part, const unsigned char* tile_todo, int* launches)
{
    if (effective_schur_path(c) == PBA_SCHUR_TENSOR)
        return launch_schur_tc(pb, Hfd, Hnn, schur_tc_lists(c), schur_lists(c), red, red_stride, c->d.Soff,
                               c->d.err, c->stream, launches);
    return launch_schur_sparse(pb, Hfd, Hnn, schur_lists(c), part, c->d.Soff, c->stream, launches, tile_todo);
}

// Places the Schur pair items of every bundle (bundle_pair_items; once per
// structure) and uploads them into the workspace: before the SIMT path
// first runs on a workspace (the tensor-core path does not read them).
pba_status fill_pair_items(pba_ctx* ctx)
{
    if (!ctx->items_ready) {
        ctx->pair_items.resize((size_t)ctx->n_pair_items);
        std::vector<int64_t> cnt;
        for (const BundleIn& b : ctx->bun) bundle_pair_items(ctx, b, cnt, ctx->pair_items.data() + b.item0);
        ctx->items_ready = true;
    }
    CK(h2d(ctx, ctx->d.pair_items, ctx->pair_items.data(), sizeof(int2) * ctx->pair_items.size()));
    return PBA_OK;
}

SolveArgs make_solve(pba_ctx* c)
{
    SolveArgs a{};
    a.F = c->F;
    a.n6 = c->n6max;
    a.B = c->B;
    a.Fmax = c->Fmax;
    a.bund = c->d.bund;
    a.frame_bundle = c->d.frame_bundle;
    a.pat = c->d.pat;
    a.P = (int)c->pattern.size() / 2;
    a.fx = c->K[0];
    a.fy = c->K[1];
    a.inv_fx = 1.0 / c->K[0];
    a.inv_fy = 1.0 / c->K[1];
    a.poses64 = c->d.poses64;
    a.poses0 = c->d.poses0_64;
    a.dtheta64 = c->d.dtheta64;
    a.dth2 = c->d.dth2;
    a.fc = c->d.fc;
    a.fc_prev = c->d.fc_prev;
    a.dthsq = c->d.dthsq;
    a.err = c->d.err;
    if (joint_brightness(c)) {
        a.dab64 = c->d.dab64;
        a.dab2 = c->d.dab2;
        a.red_aff = c->d.red_aff;
        a.photo_prior = c->cfg.photo_prior;
    }
    return a;
}

BundleSet bundle_set(pba_ctx* c)
{
    BundleSet bs{};
    bs.B = c->B;
    bs.bund = c->d.bund;
    bs.n6max = c->n6max;
    bs.nb = 6;
    return bs;
}

// The 8 (F - 1) system of the brightness pairs as unknowns (one bundle; its
// arrays start at offset 0 of the A8 / L8 / Linv8 / pivot / S8^-1 buffers).
BundleSet bundle_set8(pba_ctx* c)
{
    BundleSet b8{};
    b8.B = 1;
    b8.one = c->bdesc[0];
    b8.one.so = b8.one.ao = b8.one.lo = 0;
    b8.one.po = 0;
    b8.n6max = c->n6max;
    b8.nb = 8;
    return b8;
}

pba_status copy_stats(pba_ctx* ctx, int n_iters, pba_iter_stats* stats)
{
    pba_status s = check_device_error(ctx);
    if (s != PBA_OK) return s;
    if (!stats) return PBA_OK;
    std::vector<double> h((size_t)(n_iters + 1) * kStats);
    CK(d2h(ctx, h.data(), ctx->d.stats, sizeof(double) * h.size()));
    for (int k = 0; k <= n_iters; ++k) {
        const double* r = h.data() + (size_t)k * kStats;
        // slots hold raw sums: energy, sum r^2, count, max displacement,
        // sum |Dtheta|^2, sum Dd^2
        stats[k] = pba_iter_stats{r[0], r[2] > 0 ? std::sqrt(r[1] / r[2]) : 0.0, r[2],
                                  k < n_iters ? r[3] : 0.0, k < n_iters ? std::sqrt(r[4]) : 0.0,
                                  k < n_iters ? std::sqrt(r[5]) : 0.0};
    }
    return PBA_OK;
}

// Runs `body` (which enqueues kernels on ctx->stream) directly, or, with
// cfg.use_graphs and a non-null stream, replays it from a graph captured on
// the first call with this key. The kernels read all state from the
// workspace, so a replay computes exactly what the direct launches would.
template <class Fn>
pba_status run_enqueued(pba_ctx* ctx, GraphKey key, Fn&& body)
{
    if (!ctx->cfg.use_graphs || !ctx->stream) return body();
    auto it = ctx->graphs.find(key);
    if (it == ctx->graphs.end()) {
        GraphRec rec;
        std::vector<TimedPair> saved;
        saved.swap(ctx->tev);
        const int64_t l0 = ctx->launches;
        CK(cudaStreamBeginCapture(ctx->stream, cudaStreamCaptureModeThreadLocal));
        ctx->capturing = true;
        pba_status s = body();
        ctx->capturing = false;
        cudaGraph_t g = nullptr;
        const cudaError_t e = cudaStreamEndCapture(ctx->stream, &g);
        rec.tev.swap(ctx->tev);
        ctx->tev.swap(saved);
        rec.launches = ctx->launches - l0;
        ctx->launches = l0;
        cudaError_t ei = cudaSuccess;
        if (s == PBA_OK && e == cudaSuccess) ei = cudaGraphInstantiate(&rec.exec, g, 0);
        if (g) cudaGraphDestroy(g);
        if (s != PBA_OK || e != cudaSuccess || ei != cudaSuccess) {
            for (auto& ev : rec.tev) {
                ctx->evpool.push_back(ev.second.first);
                ctx->evpool.push_back(ev.second.second);
            }
            if (s != PBA_OK) return s;
            return fail(ctx, PBA_ERR_CUDA, "graph capture failed: %s",
                        cudaGetErrorString(e != cudaSuccess ? e : ei));
        }
        it = ctx->graphs.emplace(key, std::move(rec)).first;
    }
    CK(cudaGraphLaunch(it->second.exec, ctx->stream));
    ctx->launches += it->second.launches;
    ctx->tev_graph.insert(ctx->tev_graph.end(), it->second.tev.begin(), it->second.tev.end());
    return PBA_OK;
}

}  // namespace

namespace pba {

// Setup: central-difference gradient images (FC) and the template
// intensities of every (point, pattern pixel).
template <int DT>
__global__ void gradient_images_kernel(DevProblem pb, float* gx, float* gy)
{
    // blockIdx.z = frame (strided over gridDim.z), blockIdx.y = row, threads
    // along the row: no index divisions, coalesced rows
    const int x = blockIdx.x * blockDim.x + threadIdx.x, y = blockIdx.y;
    if (x >= pb.W) return;
    for (int f = blockIdx.z; f < pb.F; f += gridDim.z) {
        const size_t row = ((size_t)f * pb.H + y) * pb.pitch;
        float a = 0.0f, b = 0.0f;
        if (x >= 1 && x <= pb.W - 2)
            a = 0.5f * (load_px_t<DT>(pb.img, (unsigned)(row + x + 1)) -
                        load_px_t<DT>(pb.img, (unsigned)(row + x - 1)));
        if (y >= 1 && y <= pb.H - 2)
            b = 0.5f * (load_px_t<DT>(pb.img, (unsigned)(row + pb.pitch + x)) -
                        load_px_t<DT>(pb.img, (unsigned)(row - pb.pitch + x)));
        const size_t i = ((size_t)f * pb.H + y) * pb.W + x;
        gx[i] = a;
        gy[i] = b;
    }
}

// Template intensities and gradients (central differences of the reference
// image, read from the gradient images) at every pattern pixel, laid out
// [tile][j][lane]; tile t's reference image is frame tile_f0[t].
__global__ void template_gather_kernel(DevProblem pb, const int* tile_f0, float* I0p, float2* G0p)
{
    const int total = pb.T * pb.P * kTile;
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < total; i += gridDim.x * blockDim.x) {
        const int lane = i % kTile, j = (i / kTile) % pb.P, t = i / (kTile * pb.P);
        const int n = t * kTile + lane;
        const size_t row0 = (size_t)tile_f0[t] * pb.H;
        const int px = pb.uvs[2 * n] + pb.pat[2 * j], py = pb.uvs[2 * n + 1] + pb.pat[2 * j + 1];
        I0p[i] = load_px(pb.img, pb.dtype, (row0 + py) * pb.pitch + px);
        const size_t g = (row0 + py) * pb.W + px;
        G0p[i] = make_float2(pb.gx[g], pb.gy[g]);
    }
}

cudaError_t launch_setup(const DevProblem& pb, const int* tile_f0, float* gx, float* gy, float* I0p,
                         float2* G0p, cudaStream_t st)
{
    const dim3 grid((pb.W + 255) / 256, pb.H, std::min(pb.F, 65535));
    if (pb.dtype == PBA_F32) gradient_images_kernel<PBA_F32><<<grid, 256, 0, st>>>(pb, gx, gy);
    else if (pb.dtype == PBA_F16) gradient_images_kernel<PBA_F16><<<grid, 256, 0, st>>>(pb, gx, gy);
    else gradient_images_kernel<PBA_BF16><<<grid, 256, 0, st>>>(pb, gx, gy);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    template_gather_kernel<<<256, 256, 0, st>>>(pb, tile_f0, I0p, G0p);
    return cudaGetLastError();
}

}  // namespace pba

// ===========================================================================
// C ABI
// ===========================================================================
extern "C" {

pba_status pba_create(const pba_config* cfg, pba_ctx** out)
{
    if (!out) return PBA_ERR_ARG;
    *out = nullptr;
    if (!cfg || !(cfg->huber_k > 0.0) || cfg->pattern_size < 1 ||
        cfg->pattern_size > PBA_MAX_PATTERN || !cfg->pattern || cfg->n_bundles < 0 ||
        cfg->n_bundles > PBA_MAX_BUNDLES ||
        cfg->gauge_anchor_w < 0.0 || cfg->max_stats_iters < 0 || !(cfg->damping >= 0.0) ||
        !(cfg->damping < 1e6) || cfg->photometric < 0 || cfg->photometric > 2 ||
        !(cfg->photo_prior >= 0.0) || !(cfg->photo_prior < 1e12) ||
        (cfg->photometric == 2 && cfg->n_bundles > 1))
        return PBA_ERR_ARG;
    for (int j = 0; j < 2 * cfg->pattern_size; ++j)
        if (cfg->pattern[j] < -32 || cfg->pattern[j] > 32) return PBA_ERR_ARG;
    pba_ctx* c = new (std::nothrow) pba_ctx();
    if (!c) return PBA_ERR_NOMEM;
    c->cfg = *cfg;
    c->pattern.assign(cfg->pattern, cfg->pattern + 2 * cfg->pattern_size);
    c->cfg.pattern = nullptr;
    if (c->cfg.gauge_anchor_w == 0.0) c->cfg.gauge_anchor_w = 1.0;
    if (c->cfg.conv_px == 0.0) c->cfg.conv_px = 5e-3;
    if (c->cfg.max_stats_iters == 0) c->cfg.max_stats_iters = 256;
    c->stream = (cudaStream_t)cfg->cuda_stream;
    c->stats_slots = c->cfg.max_stats_iters + 1;
    c->B = std::max(1, cfg->n_bundles);
    c->cfg.n_bundles = c->B;
    c->bun.resize(c->B);
    *out = c;
    return PBA_OK;
}

void pba_destroy(pba_ctx* ctx)
{
    if (!ctx) return;
    cudaStreamSynchronize(ctx->stream);
    destroy_graphs(ctx);
    tcollect(ctx);
    for (cudaEvent_t e : ctx->evpool) cudaEventDestroy(e);
    delete ctx;
}

const char* pba_last_error(const pba_ctx* ctx) { return ctx ? ctx->err.c_str() : "null context"; }

pba_status pba_set_frames(pba_ctx* ctx, int bundle, int n_frames, int w, int h, int pitch_elems,
                          pba_dtype dtype, pba_memory mem, const void* images,
                          const double* poses, const double* intrinsics)
{
    if (!ctx) return PBA_ERR_ARG;
    if (bundle < 0 || bundle >= ctx->B)
        return fail(ctx, PBA_ERR_ARG, "bundle %d out of range (%d bundles)", bundle, ctx->B);
    if (n_frames < 2 || w < 4 || h < 4 || pitch_elems < w || !images || !poses || !intrinsics)
        return fail(ctx, PBA_ERR_ARG, "invalid frame arguments");
    if (dtype != PBA_F32 && dtype != PBA_F16 && dtype != PBA_BF16)
        return fail(ctx, PBA_ERR_ARG, "invalid dtype");
    if (mem != PBA_MEM_DEVICE && mem != PBA_MEM_HOST) return fail(ctx, PBA_ERR_ARG, "invalid memory kind");
    if (n_frames > 1024) return fail(ctx, PBA_ERR_ARG, "at most 1024 frames per bundle");
    if ((double)n_frames * h * pitch_elems >= 4294967296.0)
        return fail(ctx, PBA_ERR_ARG, "image stack too large (F * h * pitch must stay below 2^32)");
    if (mem == PBA_MEM_DEVICE && ((uintptr_t)images % elem_size(dtype)))
        return fail(ctx, PBA_ERR_ARG, "misaligned image pointer");
    for (int i = 0; i < 4; ++i)
        if (!std::isfinite(intrinsics[i])) return fail(ctx, PBA_ERR_ARG, "non-finite intrinsics");
    if (!(intrinsics[0] > 0 && intrinsics[1] > 0)) return fail(ctx, PBA_ERR_ARG, "focal lengths must be positive");
    for (int i = 0; i < 12 * n_frames; ++i)
        if (!std::isfinite(poses[i])) return fail(ctx, PBA_ERR_ARG, "non-finite pose");
    static const double I12[12] = {1, 0, 0, 0, 1, 0, 0, 0, 1, 0, 0, 0};
    for (int i = 0; i < 12; ++i)
        if (std::fabs(poses[i] - I12[i]) > 1e-9) return fail(ctx, PBA_ERR_ARG, "frame 0 pose must be the identity");
    // the bundles of a context share one camera
    for (int o = 0; o < ctx->B; ++o) {
        if (o == bundle || !ctx->bun[o].have_frames) continue;
        if (w != ctx->W || h != ctx->H || pitch_elems != ctx->pitch || dtype != ctx->dtype || mem != ctx->mem ||
            std::memcmp(intrinsics, ctx->K, sizeof ctx->K) != 0)
            return fail(ctx, PBA_ERR_ARG,
                        "bundle %d: the bundles of a context share image size, pitch, type, memory kind "
                        "and intrinsics", bundle);
    }
    BundleIn& b = ctx->bun[bundle];
    if (b.have_points && (w != ctx->W || h != ctx->H)) b.have_points = false;  // revalidate the points
    b.F = n_frames;
    b.images = images;
    b.poses_init.assign(poses, poses + 12 * n_frames);
    b.have_frames = true;
    if (b.have_points && b.F_pts != n_frames) b.have_points = false;  // entries formed for another F
    ctx->W = w;
    ctx->H = h;
    ctx->pitch = pitch_elems;
    ctx->dtype = dtype;
    ctx->mem = mem;
    std::memcpy(ctx->K, intrinsics, sizeof ctx->K);
    ctx->built = false;
    ctx->ws_ready = ctx->ic_ready = false;
    return PBA_OK;
}

pba_status pba_set_points(pba_ctx* ctx, int bundle, int n_points, const int32_t* uv,
                          const double* inv_depth, const uint8_t* vis)
{
    if (!ctx) return PBA_ERR_ARG;
    if (bundle < 0 || bundle >= ctx->B)
        return fail(ctx, PBA_ERR_ARG, "bundle %d out of range (%d bundles)", bundle, ctx->B);
    BundleIn& b = ctx->bun[bundle];
    if (!b.have_frames) return fail(ctx, PBA_ERR_STATE, "pba_set_frames must come first");
    if (n_points < 1 || !uv || !inv_depth) return fail(ctx, PBA_ERR_ARG, "invalid point arguments");
    int rad = 0;
    for (int32_t o : ctx->pattern) rad = std::max(rad, std::abs(o));
    rad += 1;  // central differences of the template
    for (int n = 0; n < n_points; ++n) {
        const int u = uv[2 * n], v = uv[2 * n + 1];
        if (u - rad < 0 || u + rad > ctx->W - 1 || v - rad < 0 || v + rad > ctx->H - 1)
            return fail(ctx, PBA_ERR_ARG, "point %d: pattern leaves the reference image", n);
        if (!(inv_depth[n] > 0.0) || !std::isfinite(inv_depth[n]))
            return fail(ctx, PBA_ERR_ARG, "point %d: inverse depth must be positive", n);
    }
    b.N = n_points;
    b.uv.assign(uv, uv + 2 * n_points);
    b.d_init.assign(inv_depth, inv_depth + n_points);
    form_tiles(b, vis);
    b.have_points = true;
    ctx->built = false;
    ctx->ws_ready = ctx->ic_ready = false;
    return PBA_OK;
}

pba_status pba_workspace_size(pba_ctx* ctx, size_t* bytes)
{
    if (!ctx || !bytes) return PBA_ERR_ARG;
    pba_status s = ensure_structure(ctx);
    if (s != PBA_OK) return s;
    *bytes = layout(ctx, nullptr);
    return PBA_OK;
}

pba_status pba_set_workspace(pba_ctx* ctx, void* dev_ptr, size_t bytes)
{
    if (!ctx) return PBA_ERR_ARG;
    pba_status st = ensure_structure(ctx);
    if (st != PBA_OK) return st;
    const size_t need = layout(ctx, nullptr);
    if (!dev_ptr || bytes < need)
        return fail(ctx, PBA_ERR_NOMEM, "workspace of %zu bytes needed, %zu given", need, bytes);
    if ((uintptr_t)dev_ptr % kAlign) return fail(ctx, PBA_ERR_ARG, "workspace must be 256-byte aligned");
    destroy_graphs(ctx);  // captured kernels hold the old workspace's pointers
    ctx->ws = (char*)dev_ptr;
    ctx->ws_bytes = bytes;
    layout(ctx, ctx->ws);
    ctx->ic_ready = false;
    CK(cudaMemsetAsync(ctx->ws, 0, need, ctx->stream));
    if (own_images(ctx)) {
        const size_t fbytes = (size_t)ctx->H * ctx->pitch * elem_size(ctx->dtype);
        for (const BundleIn& b : ctx->bun) {
            char* dst = static_cast<char*>(ctx->d.img) + fbytes * b.fo;
            if (ctx->mem == PBA_MEM_HOST) CK(h2d(ctx, dst, b.images, fbytes * b.F));
            else CK(cudaMemcpyAsync(dst, b.images, fbytes * b.F, cudaMemcpyDeviceToDevice, ctx->stream));
        }
    }
    const int Np = ctx->Npad;
    std::vector<int> uvs(2 * Np);
    std::vector<float2> xn(Np);
    std::vector<unsigned char> valid(Np, 0);
    std::vector<int> slot_caller(Np, -1);
    for (const BundleIn& b : ctx->bun) {
        // the real points fill the first N slots; a pad copies the last real
        // point (ranges of slots on the host pool)
        if (b.perm.empty()) continue;
        const int last = b.perm[b.N - 1];
        parallel_ranges((int64_t)b.perm.size(), 8192, 16, [&](int, int64_t k0, int64_t k1) {
            for (int64_t k = k0; k < k1; ++k) {
                const size_t i = (size_t)kTile * b.to + k;
                const int n = b.perm[k] >= 0 ? b.perm[k] : last;
                uvs[2 * i] = b.uv[2 * n];
                uvs[2 * i + 1] = b.uv[2 * n + 1];
                xn[i] = make_float2((float)((uvs[2 * i] - ctx->K[2]) / ctx->K[0]),
                                    (float)((uvs[2 * i + 1] - ctx->K[3]) / ctx->K[1]));
                valid[i] = b.perm[k] >= 0;
                slot_caller[i] = b.perm[k];
            }
        });
    }
    std::vector<int> pat(ctx->pattern.begin(), ctx->pattern.end());
    CK(h2d(ctx, ctx->d.pat, pat.data(), sizeof(int) * pat.size()));
    CK(h2d(ctx, ctx->d.entries, ctx->entries.data(), sizeof(Entry) * ctx->entries.size()));
    ctx->frame_on.assign(ctx->F, 1);
    ctx->frame_todo.assign(ctx->F, 0);
    ctx->frame_changed.assign(ctx->F, 0);
    ctx->window_dirty = false;
    CK(h2d(ctx, ctx->d.tile_entry, ctx->tile_entry.data(), sizeof(int) * ctx->tile_entry.size()));
    CK(h2d(ctx, ctx->d.frame_entry, ctx->frame_entry.data(), sizeof(int) * ctx->frame_entry.size()));
    CK(h2d(ctx, ctx->d.entry_slot, ctx->entry_slot.data(), sizeof(int) * ctx->entry_slot.size()));
    CK(h2d(ctx, ctx->d.frame_bundle, ctx->frame_bundle.data(), sizeof(int) * ctx->frame_bundle.size()));
    CK(h2d(ctx, ctx->d.tile_f0, ctx->tile_f0.data(), sizeof(int) * ctx->tile_f0.size()));
    CK(h2d(ctx, ctx->d.bund, ctx->bdesc.data(), sizeof(BundleDesc) * ctx->bdesc.size()));
    CK(h2d(ctx, ctx->d.uvs, uvs.data(), sizeof(int) * uvs.size()));
    CK(h2d(ctx, ctx->d.xn, xn.data(), sizeof(float2) * xn.size()));
    CK(h2d(ctx, ctx->d.valid_pt, valid.data(), valid.size()));
    CK(h2d(ctx, ctx->d.slot_caller, slot_caller.data(), sizeof(int) * slot_caller.size()));
    CK(h2d(ctx, ctx->d.pair_fg, ctx->pair_fg.data(), sizeof(int) * ctx->pair_fg.size()));
    CK(h2d(ctx, ctx->d.pair_chunk, ctx->pair_chunk.data(), sizeof(int) * ctx->pair_chunk.size()));
    CK(h2d(ctx, ctx->d.chunk_pair, ctx->chunk_pair.data(), sizeof(int) * ctx->chunk_pair.size()));
    CK(h2d(ctx, ctx->d.chunk_start, ctx->chunk_start.data(), sizeof(int) * ctx->chunk_start.size()));
    CK(h2d(ctx, ctx->d.st_info, ctx->st_info.data(), sizeof(int4) * ctx->st_info.size()));
    CK(h2d(ctx, ctx->d.st_items, ctx->st_items.data(), sizeof(int4) * ctx->st_items.size()));
    CK(h2d(ctx, ctx->d.st_rows, ctx->st_rows.data(), sizeof(StRow) * ctx->st_rows.size()));
    ctx->ic_chunks_valid = false;
    for (int bi = 0; bi < ctx->B; ++bi) {
        const BundleIn& b = ctx->bun[bi];
        pba_status s = upload_params(ctx, bi, b.poses_init.data(), b.d_init.data(), 1);
        if (s != PBA_OK) return s;
        CK(h2d(ctx, ctx->d.poses0_64 + (size_t)12 * b.fo, b.poses_init.data(), sizeof(double) * 12 * b.F));
    }
    LaunchCtx L = make_launch(ctx);
    CK(ldl_setup());
    CK(iter_setup());
    CK(linalg_setup());
    if (joint_brightness(ctx)) CK(affine_setup());
    CK(schur_tc_setup());
    {
        int dev = 0;
        CK(cudaGetDevice(&dev));
        CK(cudaDeviceGetAttribute(&ctx->n_sm, cudaDevAttrMultiProcessorCount, dev));
    }
    LAUNCH(TS_PRE, launch_setup(L.pb, ctx->d.tile_f0, ctx->d.gx, ctx->d.gy, ctx->d.I0p, ctx->d.G0p, ctx->stream));
    if (effective_schur_path(ctx) == PBA_SCHUR_SIMT) {
        pba_status s = fill_pair_items(ctx);
        if (s != PBA_OK) return s;
    }
    CK(cudaStreamSynchronize(ctx->stream));
    ctx->ws_ready = true;
    return PBA_OK;
}

pba_status precompute_core(pba_ctx* ctx, const LaunchCtx& L, const BundleSet& bs,
                           const unsigned char* todo = nullptr, const unsigned char* tile_todo = nullptr);

// The IC precompute's launches (Sec. 3.5): p_0 from the current parameters,
// J, W_0 and the H blocks per entry, the frame sums, the Schur complement, S
// with the gauge prior, its LDL^T factor and S^-1.
pba_status precompute_body(pba_ctx* ctx)
{
    const int F = ctx->F;
    LaunchCtx L = make_launch(ctx);
    const BundleSet bs = bundle_set(ctx);
    // the current parameters become p_0
    CK(cudaMemcpyAsync(ctx->d.poses0_64, ctx->d.poses64, sizeof(double) * 12 * F, cudaMemcpyDeviceToDevice,
                       ctx->stream));
    CK(cudaMemcpyAsync(ctx->d.d0_64, ctx->d.d64, sizeof(double) * ctx->Npad, cudaMemcpyDeviceToDevice,
                       ctx->stream));
    LAUNCH(TS_PRE, launch_depth_update(L, make_solve(ctx), true, 0));  // FP32 depths of p_0
    return precompute_core(ctx, L, bs);
}

// The precompute after the FP32 depths of the new p_0 are in place; with
// todo, the entries of the frames flagged there only, and with tile_todo the
// Schur chunks of the tiles flagged there only (a window update: the other
// chunks' sums are kept from the last precompute, their inputs unchanged).
pba_status precompute_core(pba_ctx* ctx, const LaunchCtx& L, const BundleSet& bs, const unsigned char* todo,
                           const unsigned char* tile_todo)
{
    LAUNCH(TS_PRE, launch_ic_precompute(L, todo));
    LAUNCH(TS_PRE, launch_frame_reduce(L, 0, 21, ctx->d.red_ic, -1, -1, true, -1, 0, ctx->d.ic_part));
    // the SIMT path keeps its chunk sums for window updates; after a
    // formation by the other path they are formed again in full
    const bool simt = effective_schur_path(ctx) == PBA_SCHUR_SIMT;
    if (simt && !ctx->ic_chunks_valid) tile_todo = nullptr;
    LAUNCHN(TS_PRE, launch_schur(ctx, L.pb, ctx->d.Hfd_ic, ctx->d.Hnn_ic, ctx->d.red_ic, 21, ctx->d.ic_schur_part,
                                 tile_todo, &nl));
    ctx->ic_chunks_valid = simt;
    LAUNCH(TS_PRE, launch_assemble_S(bs, ctx->d.red_ic, 21, ctx->d.Soff, ctx->d.poses0_64, ctx->cfg.gauge_anchor_w,
                                     ctx->cfg.damping, ctx->d.S_ic, ctx->d.active_ic, ctx->stream, ctx->d.A2,
                                     ctx->d.cmap_ic));
    if (joint_brightness(ctx)) {
        // the border of the 8 (F - 1) system, its factorisation and inverse
        // (the pose block S is the one assembled above)
        const int F = ctx->F;
        const size_t n2 = 2 * (size_t)(F - 1), n6 = 6 * (size_t)(F - 1);
        LAUNCH(TS_PRE, launch_frame_reduce(L, 0, kAffComp, ctx->d.red_aff, -1, -1, true, -1, 0,
                                           ctx->d.ic_part + kAffCol));
        CK(cudaMemsetAsync(ctx->d.aff_acc, 0, (n6 * n2 + n2 * n2) * sizeof(long long), ctx->stream));
        LAUNCH(TS_PRE, launch_affine_schur(L.pb, ctx->d.Hfd_ic, ctx->d.Had, ctx->d.Hnn_ic, ctx->d.red_ic, 21,
                                           ctx->d.red_aff, ctx->d.aff_acc, F, ctx->stream));
        LAUNCH(TS_PRE, launch_assemble_affine(ctx->d.S_ic, ctx->d.red_ic, 21, ctx->d.red_aff, ctx->d.aff_acc,
                                              ctx->d.cmap_ic, F, ctx->cfg.damping, ctx->cfg.photo_prior,
                                              ctx->d.A8, ctx->stream));
        const BundleSet b8 = bundle_set8(ctx);
        LAUNCH(TS_PRE, launch_ldl(b8, ctx->d.A8, ctx->d.L8, ctx->d.Linv8, ctx->d.dpiv8, ctx->d.rpiv8,
                                  ctx->d.cmap_ic, 0, ctx->d.err, ctx->stream, ctx->ldl_cluster));
        LAUNCH(TS_PRE, launch_ldl_inverse(b8, ctx->d.L8, ctx->d.Linv8, ctx->d.rpiv8, ctx->d.cmap_ic, ctx->d.Sinv8,
                                          ctx->stream));
        return PBA_OK;
    }
    LAUNCH(TS_PRE, launch_ldl(bs, ctx->d.A2, ctx->d.L2, ctx->d.Linv, ctx->d.dpiv, ctx->d.rpiv, ctx->d.cmap_ic, 0,
                              ctx->d.err, ctx->stream, ctx->ldl_cluster));
    LAUNCH(TS_PRE, launch_ldl_inverse(bs, ctx->d.L2, ctx->d.Linv, ctx->d.rpiv, ctx->d.cmap_ic, ctx->d.Sinv2,
                                      ctx->stream));
    return PBA_OK;
}

// FC with the brightness pairs as unknowns, after the pose system S_fc is
// assembled: the border from this iteration's H_a, the augmented 8 (F - 1)
// system, its factorisation and the backward substitution with the updates.
pba_status fc_affine_solve(pba_ctx* ctx, const LaunchCtx& L, const SolveArgs& sa)
{
    const int F = ctx->F;
    const size_t n2 = 2 * (size_t)(F - 1), n6 = 6 * (size_t)(F - 1);
    CK(cudaMemsetAsync(ctx->d.aff_acc, 0, (n6 * n2 + n2 * n2) * sizeof(long long), ctx->stream));
    LAUNCH(TS_SCHUR, launch_affine_schur(L.pb, ctx->d.Hfd_fc, ctx->d.Had_fc, ctx->d.Hnn_fc, ctx->d.red_y, 27,
                                         ctx->d.red_aff_fc, ctx->d.aff_acc, F, ctx->stream));
    LAUNCH(TS_SCHUR, launch_assemble_affine(ctx->d.S_fc, ctx->d.red_y, 27, ctx->d.red_aff_fc, ctx->d.aff_acc,
                                            ctx->d.cmap_fc, F, ctx->cfg.damping, 0.0, ctx->d.A8, ctx->stream,
                                            ctx->d.red_y, 27, 21, ctx->d.red_photo));
    const BundleSet b8 = bundle_set8(ctx);
    LAUNCH(TS_SOLVE, launch_ldl(b8, ctx->d.A8, ctx->d.L8, ctx->d.Linv8, ctx->d.dpiv8, ctx->d.rpiv8, ctx->d.cmap_fc,
                                1, ctx->d.err, ctx->stream, ctx->ldl_cluster));
    LAUNCH(TS_SOLVE, launch_fc_solve_affine(sa, ctx->d.L8, ctx->d.Linv8, ctx->stream));
    return PBA_OK;
}

// The IC solve of an iteration: Dtheta = -S^-1 y, or with the brightness
// pairs as unknowns the 8 (F - 1) system's solve and the pair update.
cudaError_t launch_ic_solve_any(pba_ctx* ctx, const SolveArgs& sa)
{
    if (joint_brightness(ctx))
        return launch_ic_solve_affine(sa, ctx->d.Sinv8, ctx->d.red_y, ctx->d.red_photo, ctx->stream);
    return launch_ic_solve(sa, ctx->d.Sinv2, ctx->d.red_y, ctx->stream);
}

// Autotuner: with the precompute's state in place, times each candidate
// launch shape on this problem (events on the context's stream, after one
// warm-up launch) and keeps the fastest. The candidates compute identical
// results, so the choice only moves time. Leaves the IC system as the
// precompute left it.
pba_status autotune(pba_ctx* ctx)
{
    cudaEvent_t a = take_event(ctx), b = take_event(ctx);
    auto elapsed = [&](auto&& launch, int reps, float* ms) -> pba_status {
        CK(launch());
        CK(cudaEventRecord(a, ctx->stream));
        for (int r = 0; r < reps; ++r) CK(launch());
        CK(cudaEventRecord(b, ctx->stream));
        CK(cudaEventSynchronize(b));
        CK(cudaEventElapsedTime(ms, a, b));
        return PBA_OK;
    };
    pba_status s = PBA_OK;
    // A candidate replaces the current shape only when it is faster by more
    // than kMargin: shapes within the timing noise of each other would
    // otherwise flip from run to run.
    constexpr float kMargin = 0.97f;
    // warps per CTA of the accumulating IC residual pass (the current shape
    // is timed first)
    float best = 0.0f;
    int best_w = ctx->res_warps;
    for (int w : {ctx->res_warps, 4, 8, 16}) {
        if (w == ctx->res_warps && best > 0.0f) continue;
        LaunchCtx L = make_launch(ctx);
        L.res_warps = w;
        float ms = 0.0f;
        s = elapsed([&]() { return launch_ic_residual(L, true, 0); }, 5, &ms);
        if (s != PBA_OK) break;
        if (best == 0.0f || ms < kMargin * best) {
            best = ms;
            best_w = w;
        }
    }
    // CTAs per bundle of the factorisation (each trial re-forms A from S);
    // the current cluster first
    const BundleSet bs = bundle_set(ctx);
    const int c0 = ctx->ldl_cluster > 0 ? ctx->ldl_cluster : ldl_max_cluster();
    int best_c = c0;
    best = 0.0f;
    std::vector<int> cands{c0};
    for (int C = 1; C <= ldl_max_cluster(); C *= 2)
        if (C != c0) cands.push_back(C);
    for (int C : cands) {
        if (s != PBA_OK) break;
        float ms = 0.0f;
        auto once = [&]() -> cudaError_t {
            cudaError_t e = launch_assemble_S(bs, ctx->d.red_ic, 21, ctx->d.Soff, ctx->d.poses0_64,
                                              ctx->cfg.gauge_anchor_w, ctx->cfg.damping, ctx->d.S_ic,
                                              ctx->d.active_ic, ctx->stream, ctx->d.A2, ctx->d.cmap_ic);
            if (e != cudaSuccess) return e;
            return launch_ldl(bs, ctx->d.A2, ctx->d.L2, ctx->d.Linv, ctx->d.dpiv, ctx->d.rpiv, ctx->d.cmap_ic, 0,
                              ctx->d.err, ctx->stream, C);
        };
        s = elapsed(once, 3, &ms);
        if (s == PBA_OK && (best == 0.0f || ms < kMargin * best)) {
            best = ms;
            best_c = C;
        }
    }
    ctx->evpool.push_back(a);
    ctx->evpool.push_back(b);
    if (s != PBA_OK) return s;
    ctx->res_warps = best_w;
    ctx->ldl_cluster = best_c;
    ctx->tuned = true;
    destroy_graphs(ctx);  // captured with the previous shapes
    return PBA_OK;
}

pba_status pba_precompute_ic(pba_ctx* ctx)
{
    if (!ctx) return PBA_ERR_ARG;
    if (!ctx->ws_ready) return fail(ctx, PBA_ERR_STATE, "workspace not set");
    if (ctx->cfg.autotune && !ctx->tuned) {
        const int timing = ctx->timing;
        ctx->timing = 0;
        pba_status s = precompute_body(ctx);
        if (s == PBA_OK) s = autotune(ctx);
        ctx->timing = timing;
        if (s != PBA_OK) return s;
    }
    pba_status s = run_enqueued(ctx, GraphKey{G_PRECOMPUTE, 0, ctx->timing},
                                [&]() -> pba_status { return precompute_body(ctx); });
    if (s != PBA_OK) return s;
    s = check_device_error(ctx);
    // a system that is not positive definite is reported (per bundle); its
    // non-positive pivots were replaced, so the other bundles of a batch can
    // iterate (that one only at the caller's risk)
    if (s == PBA_OK || s == PBA_ERR_NOT_PD) {
        ctx->ic_ready = true;
        ctx->window_dirty = false;
        std::fill(ctx->frame_todo.begin(), ctx->frame_todo.end(), 0);
        std::fill(ctx->frame_changed.begin(), ctx->frame_changed.end(), 0);
    }
    return s;
}

// Sliding window (Sec. 4.2 suggests a dynamic Hessian for windows of
// keyframes): frames leave and enter; the IC system is brought up to date
// from the stored per-entry products, precomputing only the entering frames.
pba_status pba_set_window(pba_ctx* ctx, int bundle, const uint8_t* in_window)
{
    CHECK_BUNDLE();
    if (!in_window) return fail(ctx, PBA_ERR_ARG, "null window flags");
    if (joint_brightness(ctx)) return fail(ctx, PBA_ERR_ARG, "sliding windows without the brightness unknowns");
    if (!ctx->ws_ready) return fail(ctx, PBA_ERR_STATE, "workspace not set");
    const BundleIn& b = ctx->bun[bundle];
    bool changed = false;
    for (int f = 1; f < b.F; ++f) {
        const int g = b.fo + f;
        const unsigned char on = in_window[f] != 0;
        if (on == ctx->frame_on[g]) continue;
        changed = true;
        ctx->frame_on[g] = on;
        ctx->frame_todo[g] = on;
        ctx->frame_changed[g] = 1;
        if (!on) {  // the frame's stored H_ff sums leave the frame reduction
            const int s0 = ctx->frame_entry[g], s1 = ctx->frame_entry[g + 1];
            if (s1 > s0)
                CK(cudaMemsetAsync(ctx->d.ic_part + (size_t)s0 * kEntryPartial, 0,
                                   sizeof(float) * kEntryPartial * (s1 - s0), ctx->stream));
        }
    }
    if (!changed) return PBA_OK;
    std::vector<Entry> masked(ctx->entries);
    for (Entry& e : masked)
        if (!ctx->frame_on[e.f]) e.mask = 0u;
    CK(h2d(ctx, ctx->d.entries, masked.data(), sizeof(Entry) * masked.size()));
    CK(cudaStreamSynchronize(ctx->stream));
    ctx->window_dirty = true;
    return PBA_OK;
}

pba_status pba_update_ic(pba_ctx* ctx)
{
    if (!ctx) return PBA_ERR_ARG;
    if (!ctx->ws_ready) return fail(ctx, PBA_ERR_STATE, "workspace not set");
    if (!ctx->ic_ready) return pba_precompute_ic(ctx);
    LaunchCtx L = make_launch(ctx);
    const BundleSet bs = bundle_set(ctx);
    // an entering frame is anchored at its current pose; the points keep d_0
    for (int f = 0; f < ctx->F; ++f)
        if (ctx->frame_todo[f])
            CK(cudaMemcpyAsync(ctx->d.poses0_64 + 12 * (size_t)f, ctx->d.poses64 + 12 * (size_t)f,
                               sizeof(double) * 12, cudaMemcpyDeviceToDevice, ctx->stream));
    CK(h2d(ctx, ctx->d.todo, ctx->frame_todo.data(), ctx->frame_todo.size()));
    // tiles with an entry (in or out of the window) for a frame that entered
    // or left: their points' H_dd and Schur terms change
    std::vector<unsigned char> tile_todo(ctx->T, 0);
    for (const Entry& e : ctx->entries)
        if (e.mask && ctx->frame_changed[e.f]) tile_todo[e.tile] = 1;
    CK(h2d(ctx, ctx->d.tile_todo, tile_todo.data(), tile_todo.size()));
    pba_status s = precompute_core(ctx, L, bs, ctx->d.todo, ctx->d.tile_todo);
    if (s != PBA_OK) return s;
    s = check_device_error(ctx);
    if (s == PBA_OK || s == PBA_ERR_NOT_PD) {
        ctx->window_dirty = false;
        std::fill(ctx->frame_todo.begin(), ctx->frame_todo.end(), 0);
        std::fill(ctx->frame_changed.begin(), ctx->frame_changed.end(), 0);
    }
    return s;
}

pba_status pba_iterate(pba_ctx* ctx, int n_iters, pba_iter_stats* stats)
{
    if (!ctx) return PBA_ERR_ARG;
    if (!ctx->ic_ready) return fail(ctx, PBA_ERR_STATE, "pba_precompute_ic must come first");
    if (ctx->window_dirty) return fail(ctx, PBA_ERR_STATE, "the window changed: pba_update_ic first");
    if (n_iters < 0 || n_iters > ctx->cfg.max_stats_iters)
        return fail(ctx, PBA_ERR_ARG, "n_iters must be in [0, %d]", ctx->cfg.max_stats_iters);
    LaunchCtx L = make_launch(ctx);
    SolveArgs sa = make_solve(ctx);
    sa.active = ctx->d.active_ic;
    sa.tanchor = ctx->d.poses0_64;
    sa.cmap = ctx->d.cmap_ic;
    sa.photo_sums = ctx->cfg.photometric == 1 ? ctx->d.red_photo : nullptr;
    pba_status s = run_enqueued(ctx, GraphKey{G_ITERATE, n_iters, ctx->timing}, [&]() -> pba_status {
        for (int k = 0; k < n_iters; ++k) {
            LAUNCH(TS_POINT, launch_depth_update(L, sa, true, k > 0));
            LAUNCH(TS_PASS, launch_ic_residual(L, true, k > 0));
            LAUNCH(TS_POINT, launch_ic_point(L, true));
            LAUNCH(TS_REDUCE, launch_frame_reduce(L, 0, 6, ctx->d.red_y, k, k - 1, true, 6));
            if (ctx->cfg.photometric)
                LAUNCH(TS_REDUCE, launch_frame_reduce(L, 0, 5, ctx->d.red_photo, -1, -1, true, -1, 0,
                                                      ctx->d.ent_part + kPhotoColIc));
            LAUNCH(TS_SOLVE, launch_ic_solve_any(ctx, sa));
        }
        LAUNCH(TS_EVAL, launch_depth_update(L, sa, true, n_iters > 0));
        LAUNCH(TS_EVAL, launch_ic_residual(L, false, n_iters > 0));
        LAUNCH(TS_EVAL, launch_ic_point(L, false));
        LAUNCH(TS_EVAL, launch_frame_reduce(L, 0, 0, nullptr, n_iters, n_iters - 1, false));
        return PBA_OK;
    });
    if (s != PBA_OK) return s;
    ctx->last_fc = 0;
    return copy_stats(ctx, n_iters, stats);
}

// ---------------------------------------------------------------------------
// Point sharding of one bundle (each rank a context of all frames and a share
// of the points): the halves of the IC precompute, an IC iteration and an FC
// iteration, between which the caller sums the frame sums and S_off over the
// ranks (pba_shard_export / pba_shard_import). Direct launches on the
// context's stream.
// ---------------------------------------------------------------------------
static pba_status shard_check(pba_ctx* ctx, int half)
{
    if (!ctx) return PBA_ERR_ARG;
    if (!ctx->ws_ready) return fail(ctx, PBA_ERR_STATE, "workspace not set");
    if (ctx->B != 1) return fail(ctx, PBA_ERR_ARG, "point sharding takes one bundle per context");
    if (ctx->cfg.photometric) return fail(ctx, PBA_ERR_ARG, "point sharding without the brightness model");
    if (half != 0 && half != 1) return fail(ctx, PBA_ERR_ARG, "half must be 0 or 1");
    return PBA_OK;
}

pba_status pba_shard_ic_precompute(pba_ctx* ctx, int half)
{
    pba_status s = shard_check(ctx, half);
    if (s != PBA_OK) return s;
    LaunchCtx L = make_launch(ctx);
    const BundleSet bs = bundle_set(ctx);
    if (half == 0) {
        const int F = ctx->F;
        CK(cudaMemcpyAsync(ctx->d.poses0_64, ctx->d.poses64, sizeof(double) * 12 * F, cudaMemcpyDeviceToDevice,
                           ctx->stream));
        CK(cudaMemcpyAsync(ctx->d.d0_64, ctx->d.d64, sizeof(double) * ctx->Npad, cudaMemcpyDeviceToDevice,
                           ctx->stream));
        LAUNCH(TS_PRE, launch_depth_update(L, make_solve(ctx), true, 0));
        LAUNCH(TS_PRE, launch_ic_precompute(L));
        LAUNCH(TS_PRE, launch_frame_reduce(L, 0, 21, ctx->d.red_ic, -1, -1, true, -1, 0, ctx->d.ic_part));
        LAUNCHN(TS_PRE, launch_schur(ctx, L.pb, ctx->d.Hfd_ic, ctx->d.Hnn_ic, ctx->d.red_ic, 21,
                                     ctx->d.ic_schur_part, nullptr, &nl));
        ctx->ic_chunks_valid = false;  // the kept chunk sums are this rank's only
        ctx->ic_ready = false;
        return check_device_error(ctx);
    }
    LAUNCH(TS_PRE, launch_assemble_S(bs, ctx->d.red_ic, 21, ctx->d.Soff, ctx->d.poses0_64, ctx->cfg.gauge_anchor_w,
                                     ctx->cfg.damping, ctx->d.S_ic, ctx->d.active_ic, ctx->stream, ctx->d.A2,
                                     ctx->d.cmap_ic));
    LAUNCH(TS_PRE, launch_ldl(bs, ctx->d.A2, ctx->d.L2, ctx->d.Linv, ctx->d.dpiv, ctx->d.rpiv, ctx->d.cmap_ic, 0,
                              ctx->d.err, ctx->stream, ctx->ldl_cluster));
    LAUNCH(TS_PRE, launch_ldl_inverse(bs, ctx->d.L2, ctx->d.Linv, ctx->d.rpiv, ctx->d.cmap_ic, ctx->d.Sinv2,
                                      ctx->stream));
    s = check_device_error(ctx);
    if (s == PBA_OK || s == PBA_ERR_NOT_PD) ctx->ic_ready = true;
    return s;
}

pba_status pba_shard_ic_step(pba_ctx* ctx, int k, int half)
{
    pba_status s = shard_check(ctx, half);
    if (s != PBA_OK) return s;
    if (!ctx->ic_ready) return fail(ctx, PBA_ERR_STATE, "pba_shard_ic_precompute must come first");
    if (k < 0 || k >= ctx->cfg.max_stats_iters + 1)
        return fail(ctx, PBA_ERR_ARG, "k must be in [0, %d]", ctx->cfg.max_stats_iters);
    LaunchCtx L = make_launch(ctx);
    SolveArgs sa = make_solve(ctx);
    sa.active = ctx->d.active_ic;
    sa.tanchor = ctx->d.poses0_64;
    sa.cmap = ctx->d.cmap_ic;
    if (half == 0) {
        LAUNCH(TS_POINT, launch_depth_update(L, sa, true, k > 0));
        LAUNCH(TS_PASS, launch_ic_residual(L, true, k > 0));
        LAUNCH(TS_POINT, launch_ic_point(L, true));
        LAUNCH(TS_REDUCE, launch_frame_reduce(L, 0, 6, ctx->d.red_y, k, k - 1, true, 6));
    } else {
        LAUNCH(TS_SOLVE, launch_ic_solve(sa, ctx->d.Sinv2, ctx->d.red_y, ctx->stream));
        ctx->last_fc = 0;
    }
    return PBA_OK;
}

pba_status pba_shard_fc_step(pba_ctx* ctx, int k, int half)
{
    pba_status s = shard_check(ctx, half);
    if (s != PBA_OK) return s;
    if (k < 0 || k >= ctx->cfg.max_stats_iters + 1)
        return fail(ctx, PBA_ERR_ARG, "k must be in [0, %d]", ctx->cfg.max_stats_iters);
    LaunchCtx L = make_launch(ctx);
    const BundleSet bs = bundle_set(ctx);
    SolveArgs sa = make_solve(ctx);
    sa.active = ctx->d.active_fc;
    sa.tanchor = ctx->d.poses64;
    sa.cmap = ctx->d.cmap_fc;
    if (half == 0) {
        LAUNCH(TS_POINT, launch_depth_update(L, sa, false, k > 0));
        LAUNCH(TS_PASS, launch_fc_residual(L, true, k > 0));
        LAUNCH(TS_POINT, launch_fc_point(L, true));
        LAUNCH(TS_REDUCE, launch_frame_reduce(L, 0, 27, ctx->d.red_y, k, k - 1, true, 27, 21));
        LAUNCHN(TS_SCHUR, launch_schur(ctx, L.pb, ctx->d.Hfd_fc, ctx->d.Hnn_fc, ctx->d.red_y, 27,
                                       ctx->d.schur_part, nullptr, &nl));
        return PBA_OK;
    }
    LAUNCH(TS_SCHUR, launch_assemble_S(bs, ctx->d.red_y, 27, ctx->d.Soff, ctx->d.poses64, ctx->cfg.gauge_anchor_w,
                                       ctx->cfg.damping, ctx->d.S_fc, ctx->d.active_fc, ctx->stream, ctx->d.A2,
                                       ctx->d.cmap_fc, ctx->d.red_y, 27, 21));
    LAUNCH(TS_SOLVE, launch_ldl(bs, ctx->d.A2, ctx->d.L2, ctx->d.Linv, ctx->d.dpiv, ctx->d.rpiv, ctx->d.cmap_fc, 1,
                                ctx->d.err, ctx->stream, ctx->ldl_cluster));
    LAUNCH(TS_SOLVE, launch_fc_solve_update(sa, ctx->d.L2, ctx->d.Linv, ctx->stream));
    ctx->last_fc = 1;
    return check_device_error(ctx);
}

pba_status pba_shard_eval(pba_ctx* ctx, int fc, int k)
{
    pba_status s = shard_check(ctx, 0);
    if (s != PBA_OK) return s;
    if (k < 0 || k >= ctx->cfg.max_stats_iters + 1)
        return fail(ctx, PBA_ERR_ARG, "k must be in [0, %d]", ctx->cfg.max_stats_iters);
    LaunchCtx L = make_launch(ctx);
    SolveArgs sa = make_solve(ctx);
    if (fc) {
        sa.active = ctx->d.active_fc;
        sa.tanchor = ctx->d.poses64;
        sa.cmap = ctx->d.cmap_fc;
        LAUNCH(TS_EVAL, launch_depth_update(L, sa, false, k > 0));
        LAUNCH(TS_EVAL, launch_fc_residual(L, false, k > 0));
        LAUNCH(TS_EVAL, launch_fc_point(L, false));
    } else {
        if (!ctx->ic_ready) return fail(ctx, PBA_ERR_STATE, "pba_shard_ic_precompute must come first");
        sa.active = ctx->d.active_ic;
        sa.tanchor = ctx->d.poses0_64;
        sa.cmap = ctx->d.cmap_ic;
        LAUNCH(TS_EVAL, launch_depth_update(L, sa, true, k > 0));
        LAUNCH(TS_EVAL, launch_ic_residual(L, false, k > 0));
        LAUNCH(TS_EVAL, launch_ic_point(L, false));
    }
    LAUNCH(TS_EVAL, launch_frame_reduce(L, 0, 0, nullptr, k, k - 1, false));
    return check_device_error(ctx);
}

static pba_status shard_buffer(pba_ctx* ctx, int which, double** ptr, size_t* count)
{
    const size_t F = ctx->F;
    switch (which) {
    case PBA_SHARD_IC_FRAME_SUMS: *ptr = ctx->d.red_ic; *count = F * 21; return PBA_OK;
    case PBA_SHARD_SOFF: *ptr = ctx->d.Soff; *count = (size_t)ctx->n_so; return PBA_OK;
    case PBA_SHARD_IC_RHS: *ptr = ctx->d.red_y; *count = F * 6; return PBA_OK;
    case PBA_SHARD_FC_FRAME_SUMS: *ptr = ctx->d.red_y; *count = F * 27; return PBA_OK;
    default: return fail(ctx, PBA_ERR_ARG, "unknown shard buffer %d", which);
    }
}

pba_status pba_shard_count(pba_ctx* ctx, int which, int64_t* count)
{
    if (!ctx || !count) return PBA_ERR_ARG;
    if (!ctx->ws_ready) return fail(ctx, PBA_ERR_STATE, "workspace not set");
    double* p = nullptr;
    size_t n = 0;
    pba_status s = shard_buffer(ctx, which, &p, &n);
    *count = (int64_t)n;
    return s;
}

pba_status pba_shard_export(pba_ctx* ctx, int which, double* dev_dst)
{
    if (!ctx || !dev_dst) return PBA_ERR_ARG;
    if (!ctx->ws_ready) return fail(ctx, PBA_ERR_STATE, "workspace not set");
    double* p = nullptr;
    size_t n = 0;
    pba_status s = shard_buffer(ctx, which, &p, &n);
    if (s != PBA_OK) return s;
    CK(cudaMemcpyAsync(dev_dst, p, sizeof(double) * n, cudaMemcpyDeviceToDevice, ctx->stream));
    return PBA_OK;
}

pba_status pba_shard_import(pba_ctx* ctx, int which, const double* dev_src)
{
    if (!ctx || !dev_src) return PBA_ERR_ARG;
    if (!ctx->ws_ready) return fail(ctx, PBA_ERR_STATE, "workspace not set");
    double* p = nullptr;
    size_t n = 0;
    pba_status s = shard_buffer(ctx, which, &p, &n);
    if (s != PBA_OK) return s;
    CK(cudaMemcpyAsync(p, dev_src, sizeof(double) * n, cudaMemcpyDeviceToDevice, ctx->stream));
    return PBA_OK;
}

pba_status pba_shard_stats(pba_ctx* ctx, int n_slots, double* raw)
{
    if (!ctx || !raw) return PBA_ERR_ARG;
    if (!ctx->ws_ready) return fail(ctx, PBA_ERR_STATE, "workspace not set");
    if (n_slots < 1 || n_slots > ctx->stats_slots)
        return fail(ctx, PBA_ERR_ARG, "n_slots must be in [1, %d]", ctx->stats_slots);
    std::vector<double> h((size_t)n_slots * kStats);
    CK(d2h(ctx, h.data(), ctx->d.stats, sizeof(double) * h.size()));
    for (int k = 0; k < n_slots; ++k)
        for (int q = 0; q < 6; ++q) raw[(size_t)k * 6 + q] = h[(size_t)k * kStats + q];
    return PBA_OK;
}

pba_status pba_solve_ic(pba_ctx* ctx, int n_iters, int reanchor_every, pba_iter_stats* stats)
{
    if (!ctx) return PBA_ERR_ARG;
    if (!ctx->ws_ready) return fail(ctx, PBA_ERR_STATE, "workspace not set");
    if (n_iters < 0 || n_iters > ctx->cfg.max_stats_iters || n_iters >= (1 << 16))
        return fail(ctx, PBA_ERR_ARG, "n_iters must be in [0, %d]", ctx->cfg.max_stats_iters);
    if (reanchor_every < 0 || reanchor_every >= (1 << 14))
        return fail(ctx, PBA_ERR_ARG, "reanchor_every must be in [0, 16383]");
    const int m = reanchor_every > 0 && reanchor_every < n_iters ? reanchor_every : 0;
    LaunchCtx L = make_launch(ctx);
    const BundleSet bs = bundle_set(ctx);
    SolveArgs sa = make_solve(ctx);
    sa.active = ctx->d.active_ic;
    sa.tanchor = ctx->d.poses0_64;
    sa.cmap = ctx->d.cmap_ic;
    sa.photo_sums = ctx->cfg.photometric == 1 ? ctx->d.red_photo : nullptr;
    pba_status s = run_enqueued(ctx, GraphKey{G_SOLVE, n_iters | (m << 16), ctx->timing}, [&]() -> pba_status {
        pba_status q = precompute_body(ctx);
        if (q != PBA_OK) return q;
        for (int k = 0; k < n_iters; ++k) {
            const bool reanchor = m > 0 && k > 0 && k % m == 0;
            // the step of iteration k - 1 is applied here; at a re-anchoring
            // the parameters it produces become the new p_0 and J, H, S and
            // S^-1 are formed there before the iteration's residual pass
            LAUNCH(TS_POINT, launch_depth_update(L, sa, true, k > 0));
            if (reanchor) {
                CK(cudaMemcpyAsync(ctx->d.poses0_64, ctx->d.poses64, sizeof(double) * 12 * ctx->F,
                                   cudaMemcpyDeviceToDevice, ctx->stream));
                CK(cudaMemcpyAsync(ctx->d.d0_64, ctx->d.d64, sizeof(double) * ctx->Npad, cudaMemcpyDeviceToDevice,
                                   ctx->stream));
                q = precompute_core(ctx, L, bs);
                if (q != PBA_OK) return q;
            }
            LAUNCH(TS_PASS, launch_ic_residual(L, true, k > 0));
            LAUNCH(TS_POINT, launch_ic_point(L, true));
            LAUNCH(TS_REDUCE, launch_frame_reduce(L, 0, 6, ctx->d.red_y, k, k - 1, true, 6));
            if (ctx->cfg.photometric)
                LAUNCH(TS_REDUCE, launch_frame_reduce(L, 0, 5, ctx->d.red_photo, -1, -1, true, -1, 0,
                                                      ctx->d.ent_part + kPhotoColIc));
            LAUNCH(TS_SOLVE, launch_ic_solve_any(ctx, sa));
        }
        LAUNCH(TS_EVAL, launch_depth_update(L, sa, true, n_iters > 0));
        LAUNCH(TS_EVAL, launch_ic_residual(L, false, n_iters > 0));
        LAUNCH(TS_EVAL, launch_ic_point(L, false));
        LAUNCH(TS_EVAL, launch_frame_reduce(L, 0, 0, nullptr, n_iters, n_iters - 1, false));
        return PBA_OK;
    });
    if (s != PBA_OK) return s;
    ctx->last_fc = 0;
    s = copy_stats(ctx, n_iters, stats);
    if (s == PBA_OK || s == PBA_ERR_NOT_PD) {
        ctx->ic_ready = true;
        ctx->window_dirty = false;
        std::fill(ctx->frame_todo.begin(), ctx->frame_todo.end(), 0);
        std::fill(ctx->frame_changed.begin(), ctx->frame_changed.end(), 0);
    }
    return s;
}

pba_status pba_solve_fc(pba_ctx* ctx, int n_iters, pba_iter_stats* stats)
{
    if (!ctx) return PBA_ERR_ARG;
    if (!ctx->ws_ready) return fail(ctx, PBA_ERR_STATE, "workspace not set");
    if (n_iters < 0 || n_iters > ctx->cfg.max_stats_iters)
        return fail(ctx, PBA_ERR_ARG, "n_iters must be in [0, %d]", ctx->cfg.max_stats_iters);
    LaunchCtx L = make_launch(ctx);
    const BundleSet bs = bundle_set(ctx);
    SolveArgs sa = make_solve(ctx);
    sa.active = ctx->d.active_fc;
    sa.tanchor = ctx->d.poses64;
    sa.cmap = ctx->d.cmap_fc;
    sa.photo_sums = ctx->cfg.photometric == 1 ? ctx->d.red_photo : nullptr;
    pba_status s = run_enqueued(ctx, GraphKey{G_FC, n_iters, ctx->timing}, [&]() -> pba_status {
        for (int k = 0; k < n_iters; ++k) {
            LAUNCH(TS_POINT, launch_depth_update(L, sa, false, k > 0));
            LAUNCH(TS_PASS, launch_fc_residual(L, true, k > 0));
            LAUNCH(TS_POINT, launch_fc_point(L, true));
            LAUNCH(TS_REDUCE, launch_frame_reduce(L, 0, 27, ctx->d.red_y, k, k - 1, true, 27, 21));
            if (ctx->cfg.photometric)
                LAUNCH(TS_REDUCE, launch_frame_reduce(L, 0, 5, ctx->d.red_photo, -1, -1, true, -1, 0,
                                                      ctx->d.ent_part + kPhotoColFc));
            if (joint_brightness(ctx))
                LAUNCH(TS_REDUCE, launch_frame_reduce(L, 0, kAffComp, ctx->d.red_aff_fc, -1, -1, true, -1, 0,
                                                      ctx->d.aff_part));
            LAUNCHN(TS_SCHUR, launch_schur(ctx, L.pb, ctx->d.Hfd_fc, ctx->d.Hnn_fc, ctx->d.red_y, 27,
                                           ctx->d.schur_part, nullptr, &nl));
            LAUNCH(TS_SCHUR, launch_assemble_S(bs, ctx->d.red_y, 27, ctx->d.Soff, ctx->d.poses64,
                                               ctx->cfg.gauge_anchor_w, ctx->cfg.damping, ctx->d.S_fc,
                                               ctx->d.active_fc,
                                               ctx->stream, ctx->d.A2, ctx->d.cmap_fc, ctx->d.red_y, 27, 21));
            if (joint_brightness(ctx)) {
                pba_status q = fc_affine_solve(ctx, L, sa);
                if (q != PBA_OK) return q;
                continue;
            }
            LAUNCH(TS_SOLVE, launch_ldl(bs, ctx->d.A2, ctx->d.L2, ctx->d.Linv, ctx->d.dpiv, ctx->d.rpiv,
                                        ctx->d.cmap_fc, 1, ctx->d.err, ctx->stream, ctx->ldl_cluster));
            LAUNCH(TS_SOLVE, launch_fc_solve_update(sa, ctx->d.L2, ctx->d.Linv, ctx->stream));
        }
        LAUNCH(TS_EVAL, launch_depth_update(L, sa, false, n_iters > 0));
        LAUNCH(TS_EVAL, launch_fc_residual(L, false, n_iters > 0));
        LAUNCH(TS_EVAL, launch_fc_point(L, false));
        LAUNCH(TS_EVAL, launch_frame_reduce(L, 0, 0, nullptr, n_iters, n_iters - 1, false));
        return PBA_OK;
    });
    if (s != PBA_OK) return s;
    ctx->last_fc = 1;
    return copy_stats(ctx, n_iters, stats);
}

// Device values of bundle b's point slots mapped back to the caller's point order.
static pba_status gather_points(pba_ctx* ctx, const BundleIn& b, const void* dev, bool fp32, double* out)
{
    const size_t n = b.perm.size(), off = (size_t)kTile * b.to;
    // (the scatter into caller order runs in ranges on the host pool)
    if (fp32) {
        std::vector<float> h(n);
        CK(d2h(ctx, h.data(), static_cast<const float*>(dev) + off, sizeof(float) * n));
        parallel_ranges((int64_t)n, 8192, 16, [&](int, int64_t i0, int64_t i1) {
            for (int64_t i = i0; i < i1; ++i)
                if (b.perm[i] >= 0) out[b.perm[i]] = h[i];
        });
    } else {
        std::vector<double> h(n);
        CK(d2h(ctx, h.data(), static_cast<const double*>(dev) + off, sizeof(double) * n));
        parallel_ranges((int64_t)n, 8192, 16, [&](int, int64_t i0, int64_t i1) {
            for (int64_t i = i0; i < i1; ++i)
                if (b.perm[i] >= 0) out[b.perm[i]] = h[i];
        });
    }
    return PBA_OK;
}

pba_status pba_get_params(pba_ctx* ctx, int bundle, double* poses, double* inv_depth)
{
    CHECK_BUNDLE();
    if (!ctx->ws_ready) return fail(ctx, PBA_ERR_STATE, "workspace not set");
    const BundleIn& b = ctx->bun[bundle];
    CK(cudaStreamSynchronize(ctx->stream));
    if (poses) CK(d2h(ctx, poses, ctx->d.poses64 + (size_t)12 * b.fo, sizeof(double) * 12 * b.F));
    if (inv_depth) return gather_points(ctx, b, ctx->d.d64, false, inv_depth);
    return PBA_OK;
}

pba_status pba_set_params(pba_ctx* ctx, int bundle, const double* poses, const double* inv_depth)
{
    CHECK_BUNDLE();
    if (!poses || !inv_depth) return fail(ctx, PBA_ERR_ARG, "null parameters");
    if (!ctx->ws_ready) return fail(ctx, PBA_ERR_STATE, "workspace not set");
    const BundleIn& b = ctx->bun[bundle];
    for (int i = 0; i < 12 * b.F; ++i)
        if (!std::isfinite(poses[i])) return fail(ctx, PBA_ERR_ARG, "non-finite pose");
    for (int n = 0; n < b.N; ++n)
        if (!(inv_depth[n] > 0.0) || !std::isfinite(inv_depth[n]))
            return fail(ctx, PBA_ERR_ARG, "point %d: inverse depth must be positive", n);
    return upload_params(ctx, bundle, poses, inv_depth);
}

pba_status pba_get_last_update(pba_ctx* ctx, int bundle, double* dtheta, double* dd)
{
    CHECK_BUNDLE();
    if (!ctx->ws_ready) return fail(ctx, PBA_ERR_STATE, "workspace not set");
    const BundleIn& b = ctx->bun[bundle];
    CK(cudaStreamSynchronize(ctx->stream));
    if (dtheta) CK(d2h(ctx, dtheta, ctx->d.dtheta64 + (size_t)6 * b.fo, sizeof(double) * 6 * b.F));
    if (dd) return gather_points(ctx, b, ctx->d.dd_last, false, dd);
    return PBA_OK;
}

pba_status pba_get_system(pba_ctx* ctx, int bundle, int fc, double* Hff, double* Hfd, double* Hdd,
                          double* S)
{
    CHECK_BUNDLE();
    if (!ctx->ws_ready) return fail(ctx, PBA_ERR_STATE, "workspace not set");
    if (!fc && !ctx->ic_ready) return fail(ctx, PBA_ERR_STATE, "no IC system yet");
    CK(cudaStreamSynchronize(ctx->stream));
    const BundleIn& b = ctx->bun[bundle];
    const int F = b.F, n6 = 6 * (F - 1);
    if (Hff) {
        const int stride = fc ? 27 : 21;
        std::vector<double> r((size_t)F * stride);
        CK(d2h(ctx, r.data(), (fc ? ctx->d.red_y : ctx->d.red_ic) + (size_t)b.fo * stride,
               sizeof(double) * r.size()));
        std::memset(Hff, 0, sizeof(double) * 36 * F);
        for (int f = 1; f < F; ++f) {
            int q = 0;
            for (int a = 0; a < 6; ++a)
                for (int c = a; c < 6; ++c, ++q)
                    Hff[36 * f + 6 * a + c] = Hff[36 * f + 6 * c + a] = r[(size_t)f * stride + q];
        }
    }
    if (Hfd) {
        const int64_t p0 = b.e1 > b.e0 ? ctx->entries[b.e0].pair_off : 0;
        std::vector<float> h((size_t)b.V * 6);
        CK(d2h(ctx, h.data(), (fc ? ctx->d.Hfd_fc : ctx->d.Hfd_ic) + (size_t)p0 * 6, sizeof(float) * h.size()));
        std::memset(Hfd, 0, sizeof(double) * 6 * (size_t)b.N * F);
        for (int ei = b.e0; ei < b.e1; ++ei) {
            const Entry& e = ctx->entries[ei];
            const int nvis = __builtin_popcount(e.mask);
            for (int l = 0; l < kTile; ++l) {
                if (!((e.mask >> l) & 1u)) continue;
                const int rank = __builtin_popcount(e.mask & ((1u << l) - 1u));
                const int n = b.perm[(e.tile - b.to) * kTile + l];
                for (int k = 0; k < 6; ++k)
                    Hfd[((size_t)n * F + (e.f - b.fo)) * 6 + k] =
                        h[(size_t)(e.pair_off - p0) * 6 + (size_t)k * nvis + rank];
            }
        }
    }
    if (Hdd) {
        pba_status s = gather_points(ctx, b, fc ? ctx->d.Hnn_fc : ctx->d.Hnn_ic, true, Hdd);
        if (s != PBA_OK) return s;
    }
    if (S)
        CK(d2h(ctx, S, (fc ? ctx->d.S_fc : ctx->d.S_ic) + ctx->bdesc[bundle].so, sizeof(double) * n6 * n6));
    return PBA_OK;
}

pba_status pba_num_residuals(pba_ctx* ctx, int bundle, int64_t* n)
{
    CHECK_BUNDLE();
    if (!n) return fail(ctx, PBA_ERR_ARG, "null output");
    pba_status s = ensure_structure(ctx);
    if (s != PBA_OK) return s;
    *n = ctx->bun[bundle].V * (int64_t)(ctx->pattern.size() / 2);
    return PBA_OK;
}

pba_status pba_enable_timing(pba_ctx* ctx, int mask)
{
    if (!ctx) return PBA_ERR_ARG;
    ctx->timing = mask & ((1 << TS_N) - 1);
    for (int i = 0; i < TS_N; ++i) {
        ctx->tms[i] = 0.0;
        ctx->tcount[i] = 0;
    }
    ctx->launches = 0;
    return PBA_OK;
}

pba_status pba_depth_features(pba_ctx* ctx, int bundle, float* features)
{
    CHECK_BUNDLE();
    if (!features) return fail(ctx, PBA_ERR_ARG, "null features");
    if (!ctx->ws_ready) return fail(ctx, PBA_ERR_STATE, "workspace not set");
    const BundleIn& b = ctx->bun[bundle];
    LaunchCtx L = make_launch(ctx);
    CK(launch_mlp_features(L.pb, ctx->d.fc, ctx->d.slot_caller, b.to, b.T, features, ctx->stream));
    return PBA_OK;
}

pba_status pba_propose_depths(pba_ctx* ctx, int bundle, const void* packed, float* scratch)
{
    CHECK_BUNDLE();
    if (!packed || !scratch || ((uintptr_t)packed & 15) || ((uintptr_t)scratch & 15))
        return fail(ctx, PBA_ERR_ARG, "null or misaligned network / scratch");
    if (!ctx->ws_ready) return fail(ctx, PBA_ERR_STATE, "workspace not set");
    const BundleIn& b = ctx->bun[bundle];
    LaunchCtx L = make_launch(ctx);
    float* y = scratch + (size_t)b.N * kMlpIn;
    CK(launch_mlp_features(L.pb, ctx->d.fc, ctx->d.slot_caller, b.to, b.T, scratch, ctx->stream));
    CK(launch_mlp_infer(static_cast<const uint8_t*>(packed), b.N, scratch, y, ctx->d.err, ctx->stream));
    CK(launch_mlp_propose(ctx->d.slot_caller, kTile * b.to, kTile * b.T, scratch, y, ctx->d.d64, ctx->stream));
    ctx->ic_ready = false;  // p_0 changes: the precompute must run again
    return check_device_error(ctx);
}

pba_status pba_get_brightness(pba_ctx* ctx, int bundle, double* ab)
{
    CHECK_BUNDLE();
    if (!ab) return fail(ctx, PBA_ERR_ARG, "null output");
    if (!ctx->ws_ready) return fail(ctx, PBA_ERR_STATE, "workspace not set");
    const BundleIn& b = ctx->bun[bundle];
    std::vector<float> h((size_t)b.F * kFrameConst);
    CK(d2h(ctx, h.data(), ctx->d.fc + (size_t)kFrameConst * b.fo, sizeof(float) * h.size()));
    for (int f = 0; f < b.F; ++f) {
        ab[2 * f] = h[(size_t)f * kFrameConst + kFrameAlpha];
        ab[2 * f + 1] = h[(size_t)f * kFrameConst + kFrameAlpha + 1];
    }
    return PBA_OK;
}

pba_status pba_set_brightness(pba_ctx* ctx, int bundle, const double* ab)
{
    CHECK_BUNDLE();
    if (!ab) return fail(ctx, PBA_ERR_ARG, "null pairs");
    if (!ctx->ws_ready) return fail(ctx, PBA_ERR_STATE, "workspace not set");
    const BundleIn& b = ctx->bun[bundle];
    for (int i = 0; i < 2 * b.F; ++i)
        if (!std::isfinite(ab[i])) return fail(ctx, PBA_ERR_ARG, "non-finite brightness");
    for (int f = 0; f < b.F; ++f) {
        const float v[2] = {(float)ab[2 * f], (float)ab[2 * f + 1]};
        CK(h2d(ctx, ctx->d.fc + (size_t)kFrameConst * (b.fo + f) + kFrameAlpha, v, sizeof v));
    }
    CK(cudaStreamSynchronize(ctx->stream));
    return PBA_OK;
}

pba_status pba_bundle_errors(pba_ctx* ctx, int* flags)
{
    if (!ctx || !flags) return PBA_ERR_ARG;
    for (int b = 0; b < ctx->B; ++b) flags[b] = b < (int)ctx->bundle_err.size() ? ctx->bundle_err[b] : 0;
    return PBA_OK;
}

pba_status pba_get_tuning(pba_ctx* ctx, int* res_warps, int* ldl_cluster)
{
    if (!ctx) return PBA_ERR_ARG;
    if (res_warps) *res_warps = ctx->res_warps;
    if (ldl_cluster) *ldl_cluster = ctx->ldl_cluster > 0 ? ctx->ldl_cluster : ldl_max_cluster();
    return PBA_OK;
}

pba_status pba_set_schur_path(pba_ctx* ctx, int path)
{
    if (!ctx) return PBA_ERR_ARG;
    if (path != PBA_SCHUR_TENSOR && path != PBA_SCHUR_SIMT && path != PBA_SCHUR_AUTO)
        return fail(ctx, PBA_ERR_ARG, "Schur path must be PBA_SCHUR_TENSOR, PBA_SCHUR_SIMT or PBA_SCHUR_AUTO");
    if (path != ctx->schur_path) {
        destroy_graphs(ctx);
        ctx->schur_path = path;
        ctx->ic_chunks_valid = false;
    }
    // the SIMT path reads the pair items: placed now if the workspace is
    // set (else pba_set_workspace places them)
    if (ctx->ws_ready && effective_schur_path(ctx) == PBA_SCHUR_SIMT) {
        pba_status s = fill_pair_items(ctx);
        if (s != PBA_OK) return s;
        CK(cudaStreamSynchronize(ctx->stream));
    }
    return PBA_OK;
}

pba_status pba_set_tuning(pba_ctx* ctx, int res_warps, int ldl_cluster)
{
    if (!ctx) return PBA_ERR_ARG;
    CK(ldl_setup());  // the largest co-schedulable cluster
    if (res_warps != 4 && res_warps != 8 && res_warps != 16)
        return fail(ctx, PBA_ERR_ARG, "res_warps must be 4, 8 or 16");
    if (ldl_cluster < 1 || ldl_cluster > ldl_max_cluster() || (ldl_cluster & (ldl_cluster - 1)))
        return fail(ctx, PBA_ERR_ARG, "ldl_cluster must be a power of two in [1, %d]", ldl_max_cluster());
    destroy_graphs(ctx);  // captured with the previous shapes
    ctx->res_warps = res_warps;
    ctx->ldl_cluster = ldl_cluster;
    ctx->tuned = true;
    return PBA_OK;
}

pba_status pba_transfer_bytes(pba_ctx* ctx, int64_t* h2d_out, int64_t* d2h_out)
{
    if (!ctx) return PBA_ERR_ARG;
    if (h2d_out) *h2d_out = ctx->h2d;
    if (d2h_out) *d2h_out = ctx->d2h;
    return PBA_OK;
}

pba_status pba_last_timing(pba_ctx* ctx, double* ms)
{
    if (!ctx || !ms) return PBA_ERR_ARG;
    CK(cudaStreamSynchronize(ctx->stream));
    tcollect(ctx);
    for (int i = 0; i < TS_N; ++i) ms[i] = ctx->tms[i];
    ms[TS_N] = (double)ctx->launches;
    for (int i = 0; i < TS_N; ++i) ms[TS_N + 1 + i] = (double)ctx->tcount[i];
    return PBA_OK;
}

}  // extern "C"
