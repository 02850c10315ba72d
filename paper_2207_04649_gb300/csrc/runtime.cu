// Host runtime of libdpc: planning of the grid, device memory, the order of
// the stages, the C ABI, and the batched / served job modes.
#include <algorithm>
#include <type_traits>
#include <atomic>
#include <chrono>
#include <cmath>
#include <condition_variable>
#include <cstdio>
#include <cstring>
#include <fstream>
#include <map>
#include <sstream>
#include <deque>
#include <memory>
#include <mutex>
#include <string>
#include <thread>
#include <unordered_map>
#include <vector>

#include "dpc.h"
#include "stages.cuh"

namespace dpc {

namespace {

thread_local std::string g_err;

dpc_status fail(dpc_status s, const std::string& msg) {
    g_err = msg;
    return s;
}

dpc_status cuda_fail(cudaError_t e, const char* what) {
    g_err = std::string(what) + ": " + cudaGetErrorString(e);
    return e == cudaErrorMemoryAllocation ? DPC_ERR_OOM : DPC_ERR_CUDA;
}

#define DPC_CK(call)                                                 \
    do {                                                             \
        cudaError_t e_ = (call);                                     \
        if (e_ != cudaSuccess) return cuda_fail(e_, #call);          \
    } while (0)

#define DPC_TRY(call)                                                \
    do {                                                             \
        dpc_status s_ = (call);                                      \
        if (s_ != DPC_OK) return s_;                                 \
    } while (0)

constexpr int64_t kCoordLimit = 1ll << 30;
constexpr int64_t kMaxDeltaMin = 3037000499ll;  // floor(sqrt(INT64_MAX))
constexpr uint64_t kDefaultCap = 150ull << 30;

inline size_t a256(size_t x) { return (x + 255) & ~size_t(255); }
inline int bits_for(uint64_t x) {  // smallest b with 2^b > x
    int b = 0;
    while (b < 64 && (x >> b) != 0) ++b;
    return b;
}
// S-Approx-DPC's grid side max(1, floor(eps d_cut / sqrt(d))), eps = num / den:
// the largest s with (s den)^2 d <= (num d_cut)^2, in exact 128-bit integers.
inline int64_t sapprox_side(int64_t d_cut, int32_t d, int64_t num, int64_t den) {
    const unsigned __int128 rhs = (unsigned __int128)(num * d_cut) * (unsigned __int128)(num * d_cut);
    auto fits = [&](int64_t s) {
        const unsigned __int128 t = (unsigned __int128)s * (unsigned __int128)den;
        return t * t * (unsigned)d <= rhs;
    };
    int64_t lo = 1, hi = num * d_cut / den + 1;  // fits(lo) or the side is 1; !fits(hi)
    if (!fits(lo)) return 1;
    while (hi - lo > 1) {
        const int64_t mid = lo + (hi - lo) / 2;
        (fits(mid) ? lo : hi) = mid;
    }
    return lo;
}
inline int ceil_log2(uint64_t x) {  // smallest b with 2^b >= x
    int b = 0;
    while ((1ull << b) < x) ++b;
    return b;
}

// Device bytes a batch holds, counted in stream order (every allocation and
// free of a batch is on its stream), and the most it held at once.
struct Meter {
    size_t live = 0, peak = 0;
};

// Stream-ordered device allocations released together.
struct Arena {
    cudaStream_t st = nullptr;
    Meter* meter = nullptr;  // the batch's meter, or null
    std::vector<void*> ptrs;
    size_t bytes = 0;
    cudaError_t get(void** p, size_t n) {
        n = a256(n ? n : 1);
        cudaError_t e = cudaMallocAsync(p, n, st);
        if (e == cudaSuccess) {
            ptrs.push_back(*p);
            bytes += n;
            if (meter) {
                meter->live += n;
                meter->peak = std::max(meter->peak, meter->live);
            }
        }
        return e;
    }
    template <typename T>
    cudaError_t get(T** p, size_t count) {
        return get(reinterpret_cast<void**>(p), count * sizeof(T));
    }
    void release() {
        for (void* p : ptrs) cudaFreeAsync(p, st);
        ptrs.clear();
        if (meter) meter->live -= bytes;
        bytes = 0;
    }
    // an early return frees the buffers too (stream-ordered on st)
    ~Arena() { release(); }
    Arena() = default;
    Arena(const Arena&) = delete;
    Arena& operator=(const Arena&) = delete;
};

// The device's address of memory the kernels can read and write: device
// memory, or page-locked host memory (pinned or registered); null for
// pageable host memory.
inline void* device_view(const void* p) {
    if (!p) return nullptr;
    cudaPointerAttributes a;
    if (cudaPointerGetAttributes(&a, p) != cudaSuccess) {
        cudaGetLastError();
        return nullptr;
    }
    if (a.type == cudaMemoryTypeDevice || a.type == cudaMemoryTypeManaged) return const_cast<void*>(p);
    if (a.type == cudaMemoryTypeHost) return a.devicePointer;
    return nullptr;
}

struct Input {
    const int32_t* pts;
    int64_t n;
    int32_t d;
    int64_t d_cut;
    int is_device;
};

struct Tune {
    int kch = 1024;         // candidates per dense work item
    int qch = 128;          // queries per dense work item: 128, 64 or 32 (more warps per cell)
    int kmax = 4;           // gridded dims at most
    uint32_t bf_rank = 1024;  // open points ranked below this take the brute-force pass
    int tree_warp = 2;        // tree search: 1 warp-cooperative, 0 one lane per point, 2 warp for d >= 5
    int hd_cell_factor = 2;   // datasets with d >= hd_min_d: cells of side d_cut / f searched to reach f
    int hd_min_d = 7;
    int sparse_cand = 512;    // cells of at most 4 points with more candidates than this take the dense path
    int sapprox_path = 0;     // S-Approx-DPC: 0 by the pair counts, 1 all points, 2 picks only
    int sapprox_rho_cells = 2;  // S-Approx-DPC pick path: density by cell (1), one warp per pick (0), the
                                //   dense kernels over pick items (3), 1 or 3 by the candidates per pick (2)
    int rho_bulk = 0;              // dense density kernels (d <= 4, 32-bit forms): candidates staged by bulk
                                   //   copies (cp.async.bulk) instead of 128-bit loads through registers
    int sapprox_near_threads = 2;  // S-Approx-DPC pick path: near pass one thread (1) or one warp (0) per pick,
                                   //   2 by the picks per grid cell
    int sapprox_ratio = 16;   // S-Approx-DPC: the pick path when the points' pairs exceed this many times the picks'
};

struct Batch;

}  // namespace
}  // namespace dpc

struct dpc_ctx {
    int device = 0;
    cudaStream_t stream = nullptr;
    bool own_stream = false;
    uint64_t cap = dpc::kDefaultCap;
    int debug = 0;
    int mode = 0;
    int max_inflight = 4;
    int profiling = 0;
    dpc::Tune tune;
    // jobs
    struct JobRec {
        dpc_job job;
        std::vector<int64_t> rmin, dmin;
        dpc_status status = DPC_PENDING;
        uint64_t bytes = 0;  // device footprint estimate
        std::chrono::steady_clock::time_point t_submit, t_admit, t_done;
        std::shared_ptr<dpc::Batch> kept;  // job.keep: its batch, until the result hands it out
        int kept_b = 0;                    // the job's dataset index in that batch
    };
    std::mutex mu;
    std::condition_variable cv;
    std::unordered_map<uint64_t, std::shared_ptr<JobRec>> jobs;
    std::deque<uint64_t> waiting;
    uint64_t next_ticket = 1;
    bool stop = false;
    std::vector<std::thread> workers;
    uint64_t held_bytes = 0;
    int max_batch_jobs = 64;  // served mode: jobs admitted into one batch at most
    int64_t max_batch_points = 1 << 20;  // served mode: points one batch admits at most (a larger job runs alone)
    bool has_last = false;    // last_info holds the most recent finished batch of jobs
    dpc_info last_info{};
    std::string tune_cache;   // autotuner file ("" when none)
    std::map<std::pair<int, int>, dpc::Tune> tuned;  // (largest d, log2 mean n) -> knobs
    cudaStream_t copy_stream = nullptr;  // dpc_cluster: device-to-host copies beside the compute
    cudaEvent_t copy_ev[2] = {nullptr, nullptr};
};

namespace dpc {
namespace {

// Signature of a batch for the autotuner's cache: the largest d and the
// rounded log2 of the mean n.
std::pair<int, int> tune_signature(const std::vector<Input>& in) {
    int dmax = 1;
    int64_t n = 0;
    for (const auto& x : in) {
        dmax = std::max(dmax, (int)x.d);
        n += x.n;
    }
    const double mean = in.empty() ? 1.0 : std::max(1.0, (double)n / (double)in.size());
    return {dmax, (int)std::lround(std::log2(mean))};
}

// The knobs a batch runs with: the autotuner's entry for its signature, else
// the context's.
Tune tune_for(dpc_ctx* ctx, const std::vector<Input>& in) {
    std::lock_guard<std::mutex> lk(ctx->mu);
    auto it = ctx->tuned.find(tune_signature(in));
    return it != ctx->tuned.end() ? it->second : ctx->tune;
}

std::string tune_line(const std::pair<int, int>& sig, const Tune& t) {
    std::ostringstream o;
    o << "dmax=" << sig.first << " nlog=" << sig.second << " kch=" << t.kch << " kmax=" << t.kmax
      << " bf_rank=" << t.bf_rank
      << " hd_cell_factor=" << t.hd_cell_factor << " hd_min_d=" << t.hd_min_d << " qch=" << t.qch;
    return o.str();
}

// Cache file: one tune_line per signature; unknown or malformed lines are
// skipped.
void load_tune_cache(dpc_ctx* ctx) {
    std::ifstream f(ctx->tune_cache);
    std::string line;
    while (std::getline(f, line)) {
        int dmax, nlog, kch, kmax, hf, hm, qch;
        unsigned bf;
        if (std::sscanf(line.c_str(), "dmax=%d nlog=%d kch=%d kmax=%d bf_rank=%u hd_cell_factor=%d hd_min_d=%d qch=%d",
                        &dmax, &nlog, &kch, &kmax, &bf, &hf, &hm, &qch) != 8)
            continue;
        if (kch < 32 || kch > (1 << 20) || kmax < 1 || kmax > kMaxGridDims || hf < 1 || hf > 3 || hm < 1 || hm > 9 ||
            (qch != 32 && qch != 64 && qch != 128))
            continue;
        Tune t;
        t.qch = qch;
        t.kch = kch;
        t.kmax = kmax;
        t.bf_rank = bf;
        t.hd_cell_factor = hf;
        t.hd_min_d = hm;
        ctx->tuned[{dmax, nlog}] = t;
    }
}

bool save_tune_cache(dpc_ctx* ctx) {
    std::ofstream f(ctx->tune_cache, std::ios::trunc);
    if (!f) return false;
    for (const auto& e : ctx->tuned) f << tune_line(e.first, e.second) << "\n";
    return (bool)f;
}

struct Batch {
    dpc_ctx* ctx = nullptr;
    cudaStream_t st = nullptr;
    Tune tune;  // the knobs this batch runs with (fixed when its density starts)
    int B = 0;
    int64_t N = 0;
    std::vector<DsDesc> hd;
    std::vector<int64_t> h_pt_off;
    std::vector<int64_t> h_slot_off;
    Meter meter;  // declared before the arenas, which count into it until they are released
    Arena keep, dens;
    BatchView v{};
    CellWork w{};
    DeltaBufs db{};
    DsDesc* d_desc = nullptr;
    bool has_density = false, has_rank = false;
    int dep_kind = 0;  // dependent points held: 0 none, 1 exact, 2 Approx-DPC, 3 S-Approx-DPC
    int64_t npicks = 0, nsecond = 0, sap_pairs = 0, pick_pairs = 0;  // S-Approx-DPC counters
    int density_path = 0;                                            // as dpc_info::density_path
    int grid_key_bits = 0, rank_key_bits = 0;
    // the tree over the cells, built ahead on a second stream while the ring
    // search runs (it needs the ranks only); tree_ev marks its end
    bool tree_ready = false;
    bool items_filled = false;
    CellPrepBufs item_prep{};  // the grid build's cell buffers, for fill_items
    cudaStream_t side = nullptr;
    cudaEvent_t side_ev[2] = {nullptr, nullptr};
    int32_t* rho_pub = nullptr;  // S-Approx-DPC: rho as reported (-1 where not picked)
    uint32_t class_mask = 0, dim_mask = 0;
    int64_t ncells = 0, ndense = 0, nsparse = 0, nitems = 0, ntree = 0, nbf = 0;
    int64_t cand_pairs = 0;
    int64_t tree_visits = 0, tree_pairs = 0;
    unsigned long long* d_stats = nullptr;
    uint32_t* d_counters = nullptr;  // [32] rho + [32] ring work counters
    int out_is_device = 0;
    float ms[6] = {0, 0, 0, 0, 0, 0};
    int refs = 0;
    // stage events (profiling): density 0-2 and 4, S-Approx-DPC 0-7, the
    // dependent points 8-11, labels 12-13
    cudaEvent_t ev[16] = {};
    // statistics read back at the next point where the host waits for the
    // stream anyway (no round trip of their own): 1 density, 2 dependent points
    int stats_pending = 0;
    int64_t dense_pairs = 0;
    float ms_rho_dense = 0.f;

    ~Batch() {
        if (side) cudaStreamSynchronize(side);
        keep.release();
        dens.release();
        for (auto& e : ev)
            if (e) cudaEventDestroy(e);
        for (auto& e : side_ev)
            if (e) cudaEventDestroy(e);
        if (side) cudaStreamDestroy(side);
    }

    dpc_status sync(const char* what) {
        cudaError_t e = cudaStreamSynchronize(st);
        if (e != cudaSuccess) return cuda_fail(e, what);
        return DPC_OK;
    }

    void mark(int i) {
        if (ctx->profiling) {
            if (!ev[i]) cudaEventCreate(&ev[i]);
            cudaEventRecord(ev[i], st);
        }
    }
    float elapsed(int a, int b) {
        float t = 0.f;
        if (ctx->profiling && ev[a] && ev[b]) {
            cudaEventSynchronize(ev[b]);
            cudaEventElapsedTime(&t, ev[a], ev[b]);
        }
        return t;
    }

    // Reads the device error word (the stream must be synchronized).
    dpc_status check_err(const char* stage) {
        unsigned int e = 0;
        DPC_CK(cudaMemcpy(&e, v.err, sizeof(e), cudaMemcpyDeviceToHost));
        if (e) return fail(DPC_ERR_CUDA, std::string(stage) + ": internal consistency guard tripped (code " +
                                             std::to_string(e) + ")");
        return DPC_OK;
    }

    dpc_status upload_desc() {
        DPC_CK(cudaMemcpyAsync(d_desc, hd.data(), sizeof(DsDesc) * B, cudaMemcpyHostToDevice, st));
        return DPC_OK;
    }

    // ---------------------------------------------------------- density
    dpc_status density(const std::vector<Input>& in) {
        DPC_TRY(build_grid(in));
        DPC_TRY(rho_all());
        dens.release();
        has_density = true;
        stats_pending |= 1;  // read at the next wait (settle)
        return DPC_OK;
    }

    // Reads the statistics (and the error word) of the stages that ran since
    // the last wait; one wait for the stream when any are pending.
    dpc_status settle() {
        if (!stats_pending) return DPC_OK;
        unsigned long long s8[8] = {0, 0, 0, 0, 0, 0, 0, 0};
        DPC_CK(cudaMemcpyAsync(s8, d_stats, sizeof(s8), cudaMemcpyDeviceToHost, st));
        DPC_TRY(sync("statistics"));
        const int pend = stats_pending;
        stats_pending = 0;
        if (pend & 1) {
            cand_pairs = (int64_t)(s8[0] + s8[1]);
            dense_pairs = (int64_t)s8[0];
            ms[0] = elapsed(0, 1);
            ms[1] = elapsed(1, 2);
            ms_rho_dense = elapsed(1, 4);
        }
        if (pend & 2) {
            tree_visits = (int64_t)s8[4];
            tree_pairs = (int64_t)s8[5];
            ms[2] = elapsed(8, 9);
            ms[3] = elapsed(9, 10);
            ms[4] = elapsed(10, 11);
        }
        return check_err("statistics");
    }

    // The dense cells' work items, once (the density and ring passes over
    // every point run them; S-Approx-DPC's pick path does not).
    dpc_status fill_items() {
        if (items_filled) return DPC_OK;
        DPC_CK(launch_fill_items(v, item_prep, ndense, tune.kch, st));
        items_filled = true;
        return DPC_OK;
    }

    // Local density of every point (sorted and original order).
    dpc_status rho_all() {
        DPC_TRY(fill_items());
        DPC_CK(cudaMemsetAsync(v.rho_s, 0, sizeof(int32_t) * std::max<int64_t>(N, 1), st));
        DPC_CK(cudaMemsetAsync(d_counters, 0, 64 * sizeof(uint32_t), st));
        DPC_CK(launch_rho(v, w, class_mask, nitems, nsparse, d_counters, 1 | (tune.rho_bulk ? 4 : 0), st));
        mark(4);
        DPC_CK(launch_rho(v, w, class_mask, nitems, nsparse, d_counters, 2, st));
        mark(2);
        DPC_CK(launch_rho_scatter(v, st));
        return DPC_OK;
    }

    // Uploads the inputs, plans the grid of every dataset, sorts the points
    // by cell and builds the cells, their hash table, their neighbour runs and
    // the dense work items. Leaves the temporaries in `dens` (v.in may live
    // there) for the caller to release.
    dpc_status build_grid(const std::vector<Input>& in) {
        if (!st) st = ctx->stream;
        tune = tune_for(ctx, in);
        keep.st = dens.st = st;
        keep.meter = dens.meter = &meter;
        B = (int)in.size();
        hd.assign(B, DsDesc{});
        h_pt_off.assign(B + 1, 0);
        int64_t in_total = 0, rec_total = 0;
        for (int b = 0; b < B; ++b) {
            DsDesc& ds = hd[b];
            ds.n = (int32_t)in[b].n;
            ds.d = in[b].d;
            ds.dp = ds.d <= 4 ? 1 : 2;
            ds.d_cut = in[b].d_cut;
            ds.d_cut2 = in[b].d_cut * in[b].d_cut;
            ds.pt_off = h_pt_off[b];
            ds.in_off = in_total;
            ds.rec_off = rec_total;
            h_pt_off[b + 1] = h_pt_off[b] + in[b].n;
            in_total += in[b].n * in[b].d;
            rec_total += in[b].n * ds.dp;
        }
        N = h_pt_off[B];
        if (N >= (1ll << 31)) return fail(DPC_ERR_INVALID_ARG, "batch holds 2^31 points or more");
        out_is_device = B == 1 ? in[0].is_device : 0;
        mark(0);

        // device copies of the inputs (a single device input is used in place)
        int64_t* d_pt_off = nullptr;
        DPC_CK(keep.get(&d_desc, B));
        DPC_CK(keep.get(&d_pt_off, B + 1));
        DPC_CK(cudaMemcpyAsync(d_pt_off, h_pt_off.data(), sizeof(int64_t) * (B + 1), cudaMemcpyHostToDevice, st));
        const int32_t* d_in = nullptr;
        if (B == 1 && in[0].is_device) {
            d_in = in[0].pts;
        } else {
            int32_t* buf = nullptr;
            DPC_CK(dens.get(&buf, (size_t)in_total));
            // a batch: the points the device can read (device or page-locked
            // host memory) in one gather pass, the others by one copy each
            std::vector<InJob> ij;
            for (int b = 0; b < B; ++b) {
                if (in[b].n == 0) continue;
                const void* dv = B > 1 ? (in[b].is_device ? in[b].pts : device_view(in[b].pts)) : nullptr;
                if (dv) {
                    ij.push_back({static_cast<const int32_t*>(dv), hd[b].in_off, in[b].n * in[b].d});
                    continue;
                }
                DPC_CK(cudaMemcpyAsync(buf + hd[b].in_off, in[b].pts, sizeof(int32_t) * in[b].n * in[b].d,
                                       in[b].is_device ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice, st));
            }
            if (!ij.empty()) {
                InJob* d_ij = nullptr;
                DPC_CK(dens.get(&d_ij, ij.size()));
                DPC_CK(cudaMemcpyAsync(d_ij, ij.data(), sizeof(InJob) * ij.size(), cudaMemcpyHostToDevice, st));
                DPC_CK(launch_job_inputs(d_ij, (int)ij.size(), in_total, buf, st));
            }
            d_in = buf;
        }
        v.B = B;
        v.N = N;
        v.desc = d_desc;
        v.pt_off = d_pt_off;
        v.in = d_in;

        // bounding boxes -> grid plan
        int32_t* d_mm = nullptr;
        DPC_CK(dens.get(&d_mm, (size_t)B * kMaxDims * 2));
        DPC_TRY(upload_desc());
        DPC_CK(launch_minmax(v, d_mm, st));
        std::vector<int32_t> mm((size_t)B * kMaxDims * 2);
        DPC_CK(cudaMemcpyAsync(mm.data(), d_mm, mm.size() * sizeof(int32_t), cudaMemcpyDeviceToHost, st));
        DPC_TRY(sync("bounding boxes"));
        uint64_t cbase = 0;
        h_slot_off.assign(B + 1, 0);
        for (int b = 0; b < B; ++b) {
            DsDesc& ds = hd[b];
            for (int k = 0; k < ds.d && ds.n > 0; ++k) {
                const int32_t lo = mm[(b * kMaxDims + k) * 2], hi = mm[(b * kMaxDims + k) * 2 + 1];
                if (lo < 0 || (int64_t)hi >= kCoordLimit)
                    return fail(DPC_ERR_INVALID_ARG, "coordinates must lie in [0, 2^30)");
            }
            DPC_TRY(plan(b, mm.data() + (size_t)b * kMaxDims * 2, cbase));
            class_mask |= 1u << (3 * (ds.d - 1) + ds.mode);
            dim_mask |= 1u << (ds.d - 1);
        }
        DPC_TRY(upload_desc());
        const int key_bits = bits_for(cbase > 0 ? cbase - 1 : 0);
        grid_key_bits = key_bits;
        const bool key32 = key_bits <= 32;

        // persistent per-point state
        DPC_CK(keep.get(&v.rec, (size_t)std::max<int64_t>(rec_total, 1)));
        DPC_CK(keep.get(&v.perm, N));
        v.pos_of = nullptr;  // S-Approx-DPC allocates and fills it
        DPC_CK(keep.get(&v.rho, N));
        DPC_CK(keep.get(&v.rho_s, N));
        DPC_CK(keep.get(&v.key, N));
        DPC_CK(keep.get(&v.ncells, 1));
        DPC_CK(keep.get(&v.err, 1));
        DPC_CK(cudaMemsetAsync(v.err, 0, sizeof(unsigned int), st));
        DPC_CK(keep.get(&d_stats, 8));
        DPC_CK(keep.get(&d_counters, 64));
        DPC_CK(cudaMemsetAsync(d_stats, 0, 8 * sizeof(unsigned long long), st));

        // cell keys, sort, cells
        const size_t kb = key32 ? 4 : 8;
        void *k0 = nullptr, *k1 = nullptr, *k2 = nullptr;
        uint32_t *v0 = nullptr, *v1 = nullptr, *flag = nullptr, *cidx = nullptr;
        DPC_CK(dens.get(&k0, kb * N));
        DPC_CK(dens.get(&k1, kb * N));
        DPC_CK(dens.get(&k2, kb * N));
        DPC_CK(dens.get(&v0, N));
        DPC_CK(dens.get(&v1, N));
        DPC_CK(dens.get(&flag, N));
        DPC_CK(dens.get(&cidx, N));
        void* temp = nullptr;
        const size_t temp_bytes = std::max(radix_sort_temp_bytes(N), scan_temp_bytes(N));
        DPC_CK(dens.get(&temp, temp_bytes));
        DPC_CK(keep.get(&v.cell_start, N + 1));
        DPC_CK(keep.get(&v.cell_of, N));
        DPC_CK(launch_cell_keys(v, key32, k0, v0, st));
        if (key32)
            DPC_CK(radix_sort_u32((uint32_t*)k0, v0, (uint32_t*)k2, v.perm, (uint32_t*)k1, v1, N, key_bits, temp, st));
        else
            DPC_CK(radix_sort_u64((uint64_t*)k0, v0, (uint64_t*)k2, v.perm, (uint64_t*)k1, v1, N, key_bits, temp, st));
        // block-start flags for the datasets whose runs come from the block
        // table; the cell hash serves the others (and the second ring)
        bool any_blocks = false, need_hash = false;
        for (int b = 0; b < B; ++b) {
            any_blocks |= hd[b].sbits > 0;
            need_hash |= hd[b].sbits == 0 && hd[b].n > 0;
        }
        uint32_t *bflag = nullptr, *bidx = nullptr, *d_nblocks = nullptr;
        if (any_blocks) {
            DPC_CK(dens.get(&bflag, N));
            DPC_CK(dens.get(&bidx, N));
            DPC_CK(dens.get(&d_nblocks, 1));
        }
        DPC_CK(launch_gather_cells(v, key32, k2, flag, cidx, bflag, bidx, d_nblocks, temp, st));
        uint32_t nc = 0, nblk = 0;
        if (N > 0) {
            DPC_CK(cudaMemcpyAsync(&nc, v.ncells, sizeof(uint32_t), cudaMemcpyDeviceToHost, st));
            if (any_blocks) DPC_CK(cudaMemcpyAsync(&nblk, d_nblocks, sizeof(uint32_t), cudaMemcpyDeviceToHost, st));
            DPC_TRY(sync("cell count"));
        }
        ncells = nc;

        // block table (load factor <= 1/2): 32-byte slots {key, first cell}, {occupancy}
        v.sbhash = nullptr;
        v.sbmask = 0;
        if (any_blocks && nblk > 0) {
            const int sb = ceil_log2((uint64_t)std::max<int64_t>(2 * (int64_t)nblk, 2));
            DPC_CK(keep.get(&v.sbhash, (size_t)2 << sb));
            v.sbmask = (1ull << sb) - 1;
            DPC_CK(cudaMemsetAsync(v.sbhash, 0xff, sizeof(int4) << (sb + 1), st));
            uint64_t* bkey = nullptr;
            uint32_t* bfirst = nullptr;
            unsigned long long* bocc = nullptr;
            DPC_CK(dens.get(&bkey, nblk));
            DPC_CK(dens.get(&bfirst, nblk));
            DPC_CK(dens.get(&bocc, nblk));
            DPC_CK(cudaMemsetAsync(bocc, 0, sizeof(unsigned long long) * nblk, st));
            DPC_CK(launch_blocks(v, flag, bflag, bidx, d_nblocks, nblk, bkey, bfirst, bocc, st));
        }
        // hash table of the non-empty cells (load factor <= 1/2)
        v.hash = nullptr;
        v.hmask = 0;
        if (need_hash) {
            const int hbits = ceil_log2((uint64_t)std::max<int64_t>(2 * ncells, 2));
            DPC_CK(keep.get(&v.hash, (size_t)1 << hbits));
            v.hmask = (1ull << hbits) - 1;
            DPC_CK(cudaMemsetAsync(v.hash, 0xff, sizeof(int4) << hbits, st));
            DPC_CK(launch_hash_insert(v, ncells, st));
        }

        // dense / sparse cells and the dense work items
        CellPrepBufs cb{};
        cb.dflag = flag;
        cb.sflag = cidx;
        cb.stats = d_stats;
        DPC_CK(dens.get(&cb.didx, ncells + 1));
        DPC_CK(dens.get(&cb.sidx, ncells + 1));
        DPC_CK(keep.get(&cb.dense, ncells + 1));
        DPC_CK(keep.get(&cb.sparse, ncells + 1));
        DPC_CK(keep.get(&cb.ndense, 1));
        DPC_CK(keep.get(&cb.nsparse, 1));
        DPC_CK(keep.get(&cb.nitems, 1));
        // neighbour runs of every cell, then the classes (by size and by
        // candidate count)
        int nbs = 1;
        for (int b = 0; b < B; ++b) {
            int t = 1;
            for (int j = 0; j < hd[b].k; ++j) t *= 2 * hd[b].R + 1;
            nbs = std::max(nbs, t);
        }
        cb.nbs = nbs;
        cb.qch = tune.qch;
        DPC_CK(keep.get(&cb.runs, (size_t)std::max<int64_t>(ncells, 1) * nbs));
        DPC_CK(keep.get(&cb.nruns, ncells + 1));
        DPC_CK(keep.get(&cb.cand, ncells + 1));
        uint32_t kmask = 0;
        for (int b = 0; b < B; ++b)
            kmask |= (hd[b].R == 1 && hd[b].k >= 1) ? (1u << hd[b].k) << (hd[b].sbits > 0 ? 8 : 0) : 1u;
        DPC_CK(launch_cell_runs(v, cb, ncells, kmask, st));
        DPC_CK(launch_classify_cells(v, cb, ncells, (uint32_t)tune.sparse_cand, temp, st));
        // the work items of the dense cells, counted over a bound of ncells
        // slots, so that one wait reads the classes and the items together
        DPC_CK(dens.get(&cb.nitem_c, ncells + 1));
        DPC_CK(dens.get(&cb.item_off, ncells + 1));
        DPC_CK(launch_item_prep(v, cb, ncells, tune.kch, temp, st));
        uint32_t cnts[3] = {0, 0, 0};
        if (ncells > 0) {
            DPC_CK(cudaMemcpyAsync(&cnts[0], cb.ndense, sizeof(uint32_t), cudaMemcpyDeviceToHost, st));
            DPC_CK(cudaMemcpyAsync(&cnts[1], cb.nsparse, sizeof(uint32_t), cudaMemcpyDeviceToHost, st));
            DPC_CK(cudaMemcpyAsync(&cnts[2], cb.nitems, sizeof(uint32_t), cudaMemcpyDeviceToHost, st));
            DPC_TRY(sync("cell classes and work items"));
        }
        ndense = cnts[0];
        nsparse = cnts[1];
        nitems = cnts[2];
        DPC_CK(keep.get(&cb.items, nitems + 1));
        items_filled = false;  // written by the first pass that runs them
        item_prep = cb;
        w.dense = cb.dense;
        w.ndense = cb.ndense;
        w.sparse = cb.sparse;
        w.nsparse = cb.nsparse;
        w.runs = cb.runs;
        w.nruns = cb.nruns;
        w.cand = cb.cand;
        w.items = cb.items;
        w.nitems = cb.nitems;
        w.kch = tune.kch;
        w.qch = tune.qch;
        w.nbs = nbs;
        w.stats = d_stats;
        mark(1);
        return DPC_OK;
    }

    // Grid plan of dataset b from its bounding box mm[2 * dim + {0, 1}].
    dpc_status plan(int b, const int32_t* mm, uint64_t& cbase) {
        DsDesc& ds = hd[b];
        const Tune& tn = tune;
        // cell side d_cut and reach 1: every point within d_cut lies in the 3^k
        // neighbouring cells; with factor f (datasets with d >= hd_min_d, whose
        // projection on at most 4 gridded dims lets many far points through),
        // side ceil(d_cut / f) and reach f cover the same distance more finely
        const int f = ds.d >= tn.hd_min_d ? tn.hd_cell_factor : 1;
        ds.R = f;
        ds.s = (ds.d_cut + f - 1) / f;
        // grid the dims with the most cells (a dim with one cell filters nothing)
        struct Dim {
            int dim;
            int64_t ext;
        };
        std::vector<Dim> dims;
        for (int k = 0; k < ds.d; ++k) {
            const int64_t lo = ds.n > 0 ? mm[2 * k] : 0, hi = ds.n > 0 ? mm[2 * k + 1] : 0;
            const int64_t ext = (hi - lo) / ds.s + 1;
            if (ext > 1) dims.push_back({k, ext});
        }
        std::stable_sort(dims.begin(), dims.end(), [](const Dim& a, const Dim& c) { return a.ext > c.ext; });
        int k = std::min<int>((int)dims.size(), std::min(tn.kmax, kMaxGridDims));
        int mbits = 0;
        auto mb = [&](int kk) {
            int m = 0;
            for (int j = 0; j < kk; ++j) m = std::max(m, ceil_log2((uint64_t)dims[j].ext));
            return m;
        };
        mbits = mb(k);
        while (k > 0 && k * mbits > 40) {
            --k;
            mbits = mb(k);
        }
        ds.k = k;
        ds.mbits = mbits;
        for (int j = 0; j < kMaxGridDims; ++j) {
            ds.dmask[j] = 0;
            for (int i = 0; j < k && i < mbits; ++i) ds.dmask[j] |= 1ull << (i * k + j);
        }
        for (int j = 0; j < kMaxGridDims; ++j) {
            ds.gdim[j] = j < k ? dims[j].dim : 0;
            ds.origin[j] = j < k ? mm[2 * dims[j].dim] : 0;
            ds.ext[j] = j < k ? (int32_t)dims[j].ext : 1;
        }
        ds.cbase = cbase;
        cbase += 1ull << (k * mbits);
        // the neighbour runs skip cells whose box is at least d_cut away: with
        // reach 1 a cell off in n dims is at least sqrt(n) away, with reach R
        // the farthest ring's corner cells at least sqrt(k) ((R - 1) s + 1)
        {
            const int64_t g = (int64_t)(ds.R - 1) * ds.s + 1;
            ds.prune = (int64_t)k * g * g >= ds.d_cut2 ? 1 : 0;
        }
        // 32-bit pair arithmetic when the largest possible candidate sum fits
        int64_t maxsum = 0;
        for (int c = 0; c < ds.d; ++c) {
            int64_t md = 0;
            bool gridded = false;
            for (int j = 0; j < k; ++j) gridded |= ds.gdim[j] == c;
            if (ds.n > 0) md = (int64_t)mm[2 * c + 1] - mm[2 * c];
            if (gridded) md = std::min<int64_t>(md, (int64_t)(ds.R + 1) * ds.s - 1);
            maxsum += md * md;
            if (maxsum >= (1ll << 31)) break;
        }
        ds.w32 = (maxsum < (1ll << 31) && ds.d_cut2 <= (1ll << 31)) ? 1 : 0;
        // neighbour runs from the block table (blocks of 2^(6 / k) cells per
        // dim, 2 for k = 4) unless some neighbours are left out or the reach
        // is not 1; the block key packs the dataset index above 40 bits
        ds.sbits = (ds.R == 1 && k >= 1 && !ds.prune && b < (1 << 23)) ? k * (k == 4 ? 1 : 6 / k) : 0;
        ds.rbits = bits_for((uint64_t)ds.n);
        // Expanded test in wrapping 32-bit arithmetic (d <= 4): with reach 1
        // every candidate differs from its query by less than 2s in each
        // gridded dim and by less than s in a dim narrower than one cell, so
        // |q - c|^2 - T lies in [-T, 4 d s^2) inside [-2^31, 2^31) when
        // 9 d s^2 < 2^31, and the wrapped sum's sign bit is exact.
        bool narrow = true;
        for (int c = 0; c < ds.d; ++c) {
            ds.lo[c] = ds.n > 0 ? mm[2 * c] : 0;
            ds.span[c] = ds.n > 0 ? mm[2 * c + 1] - mm[2 * c] + 1 : 1;
            bool gridded = false;
            for (int j = 0; j < k; ++j) gridded |= ds.gdim[j] == c;
            if (!gridded && ds.n > 0 && (int64_t)mm[2 * c + 1] - mm[2 * c] >= ds.s) narrow = false;
        }
        const bool expand = ds.d <= 4 && ds.R == 1 && narrow && ds.d_cut2 <= ds.s * ds.s &&
                            9 * (int64_t)ds.d * ds.s * ds.s < (1ll << 31);
        ds.mode = expand ? 2 : (ds.w32 ? 0 : 1);
        return DPC_OK;
    }

    // Allocates the cell tree's buffers (on st) and builds the tree on the
    // side stream, to overlap the ring search; open_points waits for it.
    dpc_status prebuild_tree(Arena& tmp) {
        const int64_t nc = ncells;
        if (nc == 0) return DPC_OK;
        db.ncells = nc;
        db.dpb = 1;
        db.compact = 1;
        for (int b = 0; b < B; ++b) {
            if (hd[b].dp == 2) db.dpb = 2;
            if (hd[b].d > 3) db.compact = 0;
        }
        if (nc >= (1ll << 29)) db.compact = 0;  // stacked link words must stay non-negative
        DPC_CK(tmp.get(&db.cell_off, B + 1));
        DPC_CK(tmp.get(&db.ckey, nc));
        DPC_CK(tmp.get(&db.child, nc));
        DPC_CK(tmp.get(&db.iparent, nc));
        DPC_CK(tmp.get(&db.lparent, nc));
        DPC_CK(tmp.get(&db.nodes, (size_t)2 * nc * (2 * db.dpb + 1)));
        DPC_CK(tmp.get(&db.flag, nc));
        DPC_CK(cudaMemsetAsync(db.flag, 0, sizeof(uint32_t) * std::max<int64_t>(nc, 1), st));
        if (!side) {
            DPC_CK(cudaStreamCreateWithFlags(&side, cudaStreamNonBlocking));
            for (auto& e : side_ev) DPC_CK(cudaEventCreateWithFlags(&e, cudaEventDisableTiming));
        }
        DPC_CK(cudaEventRecord(side_ev[0], st));
        DPC_CK(cudaStreamWaitEvent(side, side_ev[0], 0));
        DPC_CK(launch_tree_build(v, db, side));
        DPC_CK(cudaEventRecord(side_ev[1], side));
        tree_ready = true;
        return DPC_OK;
    }

    // The open points of db.tree_list / db.bf_list (counts in db.ucount[0..1],
    // filled by the stream's previous kernels): tree search and brute force.
    dpc_status open_points(Arena& tmp, const char* what) {
        if (tree_ready) DPC_CK(cudaStreamWaitEvent(st, side_ev[1], 0));  // the tree built ahead
        uint32_t uc[2] = {0, 0};
        DPC_CK(cudaMemcpyAsync(uc, db.ucount, sizeof(uc), cudaMemcpyDeviceToHost, st));
        DPC_TRY(sync(what));
        DPC_TRY(settle());  // the stream is idle: the density statistics cost no extra wait
        ntree = uc[0];
        nbf = uc[1];
        if (ntree > 0) {
            // neighbouring lanes should search neighbouring points: sort the
            // open list by sorted (Morton) position, unless it is in that order
            if (!db.lists_sorted) {
                uint32_t *ks = nullptr, *kt = nullptr, *vs = nullptr, *vt = nullptr;
                void* t3 = nullptr;
                DPC_CK(tmp.get(&ks, ntree));
                DPC_CK(tmp.get(&kt, ntree));
                DPC_CK(tmp.get(&vs, ntree));
                DPC_CK(tmp.get(&vt, ntree));
                DPC_CK(tmp.get(&t3, radix_sort_temp_bytes(ntree)));
                DPC_CK(radix_sort_u32(db.tree_list, db.tree_list, ks, vs, kt, vt, ntree, bits_for((uint64_t)N),
                                      t3, st));
                db.tree_list = ks;
            }
            const int64_t nc = ncells;
            db.ncells = nc;
            if (!tree_ready) {
                db.dpb = 1;
                db.compact = 1;
                for (int b = 0; b < B; ++b) {
                    if (hd[b].dp == 2) db.dpb = 2;
                    if (hd[b].d > 3) db.compact = 0;
                }
                if (nc >= (1ll << 29)) db.compact = 0;  // stacked link words must stay non-negative
                DPC_CK(tmp.get(&db.cell_off, B + 1));
                DPC_CK(tmp.get(&db.ckey, nc));
                DPC_CK(tmp.get(&db.child, nc));
                DPC_CK(tmp.get(&db.iparent, nc));
                DPC_CK(tmp.get(&db.lparent, nc));
                DPC_CK(tmp.get(&db.nodes, (size_t)2 * nc * (2 * db.dpb + 1)));
                DPC_CK(tmp.get(&db.flag, nc));
                DPC_CK(cudaMemsetAsync(db.flag, 0, sizeof(uint32_t) * std::max<int64_t>(nc, 1), st));
                DPC_CK(launch_tree_build(v, db, st));
            }
            DPC_CK(tmp.get(&db.stats, 2));
            DPC_CK(cudaMemsetAsync(db.stats, 0, 2 * sizeof(unsigned long long), st));
            db.key_bits = 1;
            for (int b = 0; b < B; ++b) db.key_bits = std::max(db.key_bits, hd[b].k * hd[b].mbits);
            DPC_CK(launch_tree_search(v, db, dim_mask, ntree, tune.tree_warp, st));
        }
        if (nbf > 0) {
            DPC_CK(tmp.get(&db.rrec, 2 * N));
            DPC_CK(tmp.get(&db.rorig, N));
            DPC_CK(launch_bruteforce(v, db, dim_mask, nbf, st));
        }
        return DPC_OK;
    }

    // The open-point statistics, kept on the device (the lists' buffers are
    // freed before they are read) and read by settle().
    dpc_status finish_stats(const char*) {
        DPC_CK(cudaMemsetAsync(d_stats + 4, 0, 3 * sizeof(unsigned long long), st));
        if (ntree > 0) {
            DPC_CK(cudaMemcpyAsync(d_stats + 4, db.stats, 2 * sizeof(unsigned long long), cudaMemcpyDeviceToDevice,
                                   st));
            DPC_CK(cudaMemcpyAsync(d_stats + 6, db.tcount, sizeof(uint32_t), cudaMemcpyDeviceToDevice, st));
        }
        stats_pending |= 2;
        return DPC_OK;
    }

    // -------------------------------------------------------- dependent
    // The rank order (rho desc, index asc) and the per-point state the
    // dependent-point passes write, once per batch.
    dpc_status ensure_rank(Arena& tmp, void* temp) {
        if (has_rank) return DPC_OK;
        DPC_CK(keep.get(&v.rank, N));
        DPC_CK(keep.get(&v.order, N));
        DPC_CK(keep.get(&v.ro_s, N));
        DPC_CK(keep.get(&v.dep, N));
        DPC_CK(keep.get(&v.delta2, N));
        DPC_CK(keep.get(&v.exact, N));
        int rbits = 1;
        for (int b = 0; b < B; ++b) rbits = std::max(rbits, hd[b].rbits);
        int bbits = ceil_log2((uint64_t)B);
        rank_key_bits = bbits + rbits;
        const size_t kb = (bbits + rbits) > 32 ? 8 : 4;
        DPC_CK(tmp.get(&db.rkeys, 3 * a256(kb * N) / 4 + 64));
        DPC_CK(tmp.get(&db.rvals, 2 * (N + 64)));
        DPC_CK(launch_rank(v, db, rbits, temp, st));
        has_rank = true;
        return DPC_OK;
    }

    dpc_status dependent() {
        if (dep_kind == 1 || dep_kind == 3) return DPC_OK;  // S-Approx-DPC keeps its own
        if (!has_density) return fail(DPC_ERR_STATE, "dataset has no density");
        mark(8);
        Arena tmp;
        tmp.st = st;
        tmp.meter = &meter;
        // on every way out, st waits for the tree built on the side stream
        // before tmp (which holds its buffers) is freed
        struct SideWait {
            Batch* b;
            ~SideWait() {
                if (b->tree_ready) cudaStreamWaitEvent(b->st, b->side_ev[1], 0);
                b->tree_ready = false;
            }
        } side_wait{this};
        void* temp = nullptr;
        DPC_CK(tmp.get(&temp, std::max(radix_sort_temp_bytes(N), scan_temp_bytes(N))));
        DPC_TRY(ensure_rank(tmp, temp));
        mark(9);

        DPC_CK(tmp.get(&v.best_s, N));
        DPC_CK(cudaMemsetAsync(v.best_s, 0xff, sizeof(unsigned long long) * std::max<int64_t>(N, 1), st));
        DPC_TRY(prebuild_tree(tmp));
        DPC_CK(launch_ring(v, w, class_mask, nitems, nsparse, d_counters + 32, st));
        mark(10);

        DPC_CK(tmp.get(&db.ucount, 4));
        DPC_CK(tmp.get(&db.tree_list, N));
        DPC_CK(tmp.get(&db.bf_list, N));
        DPC_CK(cudaMemsetAsync(db.ucount, 0, 4 * sizeof(uint32_t), st));
        db.tcount = db.ucount;
        db.bf_rank = tune.bf_rank;
        void* fin_temp = nullptr;
        DPC_CK(tmp.get(&fin_temp, finalize_temp_bytes(N)));
        DPC_CK(tmp.get(&db.tclass, kMaxDims + 1));
        DPC_CK(launch_finalize(v, db, fin_temp, st));
        db.lists_sorted = 1;  // written in position order, grouped by dimension
        DPC_TRY(open_points(tmp, "ring search"));
        db.lists_sorted = 0;
        db.tclass = nullptr;
        mark(11);
        DPC_TRY(finish_stats("dependent points"));
        tmp.release();  // after open_points, whose stream waited for the side stream's tree
        dep_kind = 1;
        return DPC_OK;
    }

    // ------------------------------------------------------- Approx-DPC
    // Approx-DPC's dependent points (Section 4.3): see approx.cu. The grid of
    // side max(1, floor(d_cut / sqrt(d))) covers all d dims; its keys pack
    // each dim's cell coordinate at its own bit offset after a per-dataset
    // base, and must fit 64 bits for the whole batch.
    dpc_status dependent_approx() {
        if (dep_kind == 2) return DPC_OK;
        if (dep_kind == 3) return fail(DPC_ERR_STATE, "an S-Approx-DPC dataset has densities of its picks only");
        if (!has_density) return fail(DPC_ERR_STATE, "dataset has no density");
        // keys: every dim's cell coordinate at its own bit offset, the
        // dataset's index above them (any width: sorted 64 bits at a time)
        int bshift = 0;
        for (int b = 0; b < B; ++b) {
            DsDesc& ds = hd[b];
            const int64_t q = ds.d_cut2 / ds.d;
            int64_t s = (int64_t)std::sqrt((double)q);
            while (s > 0 && s * s > q) --s;
            while ((s + 1) * (s + 1) <= q) ++s;
            ds.a_side = (int32_t)std::max<int64_t>(1, s);
            int off = 0;
            for (int k = 0; k < kMaxDims; ++k) {
                ds.a_shift[k] = off;
                if (k < ds.d && ds.n > 0) off += bits_for((uint64_t)((ds.span[k] - 1) / ds.a_side));
            }
            bshift = std::max(bshift, off);
        }
        const int key_bits = bshift + bits_for((uint64_t)(B - 1));
        DPC_TRY(upload_desc());
        mark(8);
        Arena tmp;
        tmp.st = st;
        tmp.meter = &meter;
        void* temp = nullptr;
        DPC_CK(tmp.get(&temp, std::max(radix_sort_temp_bytes(N), scan_temp_bytes(N))));
        DPC_TRY(ensure_rank(tmp, temp));
        mark(9);
        ApproxBufs ab{};
        uint64_t* kbuf = nullptr;
        uint32_t* obuf = nullptr;
        DPC_CK(tmp.get(&kbuf, 3 * a256(N)));
        DPC_CK(tmp.get(&obuf, 3 * a256(N)));
        DPC_CK(tmp.get(&ab.flag, N));
        DPC_CK(tmp.get(&ab.cidx, N));
        DPC_CK(tmp.get(&ab.cell_of, N));
        DPC_CK(tmp.get(&ab.start, N + 1));
        DPC_CK(tmp.get(&ab.top, N));
        DPC_CK(tmp.get(&ab.maxrank, N));
        DPC_CK(tmp.get(&ab.ncells, 1));
        DPC_CK(tmp.get(&ab.light, N));
        DPC_CK(tmp.get(&ab.heavy, N));
        DPC_CK(tmp.get(&ab.nlh, 2));
        DPC_CK(cudaMemsetAsync(ab.ncells, 0, sizeof(uint32_t), st));
        DPC_CK(cudaMemsetAsync(ab.nlh, 0, 2 * sizeof(uint32_t), st));
        DPC_CK(launch_approx_keys(v, key_bits, bshift, kbuf, obuf, temp, &ab.ord, st));
        DPC_CK(launch_approx_cells(v, w, ab, key_bits, bshift, temp, st));
        DPC_CK(tmp.get(&v.best_s, N));
        DPC_CK(cudaMemsetAsync(v.best_s, 0xff, sizeof(unsigned long long) * std::max<int64_t>(N, 1), st));
        DPC_CK(tmp.get(&db.ucount, 4));
        DPC_CK(tmp.get(&db.tree_list, N));
        DPC_CK(tmp.get(&db.bf_list, N));
        DPC_CK(cudaMemsetAsync(db.ucount, 0, 4 * sizeof(uint32_t), st));
        db.tcount = db.ucount;
        db.bf_rank = tune.bf_rank;
        DPC_CK(launch_approx_rules(v, w, ab, db, dim_mask, N, st));
        mark(10);
        DPC_TRY(open_points(tmp, "approximate rules"));
        mark(11);
        DPC_TRY(finish_stats("approximate dependent points"));
        tmp.release();
        dep_kind = 2;
        return DPC_OK;
    }

    // ------------------------------------------------------ S-Approx-DPC
    // S-Approx-DPC (Section 5): see sapprox.cu. Its grid G' covers all d
    // dims like Approx-DPC's, with side max(1, floor(eps d_cut / sqrt(d))).
    dpc_status sapprox(const std::vector<Input>& in, const std::vector<int64_t>& eps_num,
                       const std::vector<int64_t>& eps_den) {
        DPC_TRY(build_grid(in));
        DPC_CK(keep.get(&v.pos_of, N));
        DPC_CK(launch_pos_of(v, st));
        // key of G': every dim's cell coordinate at its own bit offset, the
        // dataset's index above them (any width: sorted 64 bits at a time)
        int bshift = 0;
        for (int b = 0; b < B; ++b) {
            DsDesc& ds = hd[b];
            ds.a_side = (int32_t)std::min<int64_t>(sapprox_side(ds.d_cut, ds.d, eps_num[b], eps_den[b]), 1ll << 30);
            int off = 0;
            for (int k = 0; k < kMaxDims; ++k) {
                ds.a_shift[k] = off;
                if (k < ds.d && ds.n > 0) off += bits_for((uint64_t)((ds.span[k] - 1) / ds.a_side));
            }
            bshift = std::max(bshift, off);
        }
        const int key_bits = bshift + bits_for((uint64_t)(B - 1));
        DPC_TRY(upload_desc());
        Arena tmp;
        tmp.st = st;
        tmp.meter = &meter;
        SapproxBufs sb{};
        void* temp = nullptr;
        DPC_CK(tmp.get(&temp, std::max(radix_sort_temp_bytes(N), scan_temp_bytes(N))));
        DPC_CK(tmp.get(&sb.keys, 3 * a256(N)));
        DPC_CK(tmp.get(&sb.ord, 3 * a256(N)));
        DPC_CK(tmp.get(&sb.flag, N));
        DPC_CK(tmp.get(&sb.cidx, N));
        DPC_CK(tmp.get(&sb.picks, N));
        DPC_CK(tmp.get(&sb.pick_s, N));
        DPC_CK(tmp.get(&sb.npicks, 1));
        DPC_CK(tmp.get(&sb.scan, N));
        DPC_CK(tmp.get(&sb.nscan, 1));
        DPC_CK(tmp.get(&sb.stats, 3));
        DPC_CK(keep.get(&v.pick, N));
        DPC_CK(cudaMemsetAsync(sb.npicks, 0, sizeof(uint32_t), st));
        DPC_CK(cudaMemsetAsync(sb.nscan, 0, sizeof(uint32_t), st));
        DPC_CK(cudaMemsetAsync(sb.stats, 0, 3 * sizeof(unsigned long long), st));
        DPC_CK(launch_sapprox_grid(v, sb, key_bits, bshift, temp, st));
        DPC_CK(launch_sapprox_pick_pairs(v, w, sb, N, st));
        uint32_t m = 0;
        unsigned long long cnt3[3] = {0, 0, 0}, allp[2] = {0, 0};
        DPC_CK(cudaMemcpyAsync(&m, sb.npicks, sizeof(uint32_t), cudaMemcpyDeviceToHost, st));
        DPC_CK(cudaMemcpyAsync(cnt3, sb.stats, sizeof(cnt3), cudaMemcpyDeviceToHost, st));
        DPC_CK(cudaMemcpyAsync(allp, d_stats, sizeof(allp), cudaMemcpyDeviceToHost, st));
        DPC_TRY(sync("S-Approx-DPC grid"));
        npicks = m;
        pick_pairs = (int64_t)cnt3[2];
        const int64_t all_pairs = (int64_t)(allp[0] + allp[1]);
        mark(7);

        // densities of the picks; the others get 0 and rank after every
        // pick. The all-point path (dense density kernels, then the ring
        // search over pick ranks) evaluates all_pairs candidate pairs twice
        // at a low cost per pair; the pick path (the picks' density, then
        // the first-phase scan per queued pick) evaluates pick_pairs twice
        // at a few times that cost, and both carry fixed costs per point
        // (grid, ranks, the searches for open points). Measured: at 5.8M x 3
        // with mean rho 100 (ratio 6.3) the all-point path is faster, 13.3
        // vs 15.4 ms; on the same points with mean rho in the thousands the
        // pick path is, from ratio 5.0 (eps 0.2) on.
        bool pick_items = false;
        density_path = 0;
        // With many pairs (2e10 and more) their cost outweighs the paths'
        // fixed costs and the pick path wins from a ratio of 4 (dense
        // 5.8M x 3 at eps 0.2: ratio 5.0, 80 vs 122 ms).
        const int64_t ratio = all_pairs >= 20000000000ll ? std::min<int64_t>(4, tune.sapprox_ratio) : tune.sapprox_ratio;
        const bool all_points = tune.sapprox_path == 1 || (tune.sapprox_path == 0 && pick_pairs * ratio >= all_pairs);
        if (all_points) {
            DPC_TRY(rho_all());
            DPC_CK(launch_sapprox_mask(v, st));
        } else {
            DPC_CK(cudaMemsetAsync(v.rho_s, 0, sizeof(int32_t) * std::max<int64_t>(N, 1), st));
            DPC_CK(cudaMemsetAsync(v.rho, 0, sizeof(int32_t) * std::max<int64_t>(N, 1), st));
            DPC_CK(cudaMemsetAsync(d_counters, 0, 64 * sizeof(uint32_t), st));
            // each cell's picks, contiguous: the density and the near pass
            // take them cell by cell
            DPC_CK(tmp.get(&sb.pflag, N));
            DPC_CK(tmp.get(&sb.ppos, N));
            DPC_CK(tmp.get(&sb.plist, N));
            DPC_CK(tmp.get(&sb.pstart, ncells + 1));
            DPC_CK(launch_sapprox_plist(v, sb, ncells, temp, st));
            // picks facing fewer than 512 candidates each: one warp per cell
            // stages its candidates once for all its picks; more: the dense
            // density kernels over (cell, pick chunk, candidate chunk) items,
            // up to 4 picks per lane in the exact grid's pair form
            int rho_mode = tune.sapprox_rho_cells;
            if (rho_mode == 2) rho_mode = pick_pairs < 512 * std::max<int64_t>(npicks, 1) ? 1 : 3;
            if (rho_mode == 3) {
                // items per cell <= picks x (candidates / kch + 1), so their
                // sum is at most npicks + pick_pairs / kch
                const int64_t cap = npicks + pick_pairs / tune.kch + 1;
                uint32_t *nitem_c = nullptr, *item_off = nullptr, *pn = nullptr;
                uint4* pitems = nullptr;
                DPC_CK(tmp.get(&nitem_c, std::max<int64_t>(ncells, 1)));
                DPC_CK(tmp.get(&item_off, std::max<int64_t>(ncells, 1)));
                DPC_CK(tmp.get(&pitems, cap));
                DPC_CK(tmp.get(&pn, 1));
                DPC_CK(launch_sapprox_items(v, w, sb, ncells, tune.kch, nitem_c, item_off, pitems, pn, cap, temp, st));
                CellWork wp = w;
                wp.qch = kQch;  // pick items hold up to kQch picks each
                wp.items = pitems;
                wp.nitems = pn;
                mark(4);
                DPC_CK(launch_rho_picks(v, wp, class_mask, cap, d_counters, sb.plist, sb.pstart, st));
                DPC_CK(launch_rho_scatter(v, st));
                pick_items = true;
            } else {
                DPC_CK(launch_sapprox_rho(v, w, sb, dim_mask, npicks, ncells, rho_mode == 1, st));
            }
            density_path = rho_mode == 3 ? 3 : (rho_mode == 1 ? 2 : 1);
            mark(2);
        }
        DPC_TRY(ensure_rank(tmp, temp));
        mark(5);

        // nearest higher pick of every point's searched block (the exact
        // ring search over pick ranks, when picks are many), the first
        // phase, then the second phase for the picks it leaves open
        DPC_CK(tmp.get(&v.best_s, N));
        DPC_CK(cudaMemsetAsync(v.best_s, 0xff, sizeof(unsigned long long) * std::max<int64_t>(N, 1), st));
        // with few picks every pick scans its own neighbourhood instead (the
        // scan keeps the block's nearest higher pick too): the cost follows
        // the picks, not the points
        if (all_points) DPC_CK(launch_ring(v, w, class_mask, nitems, nsparse, d_counters + 32, st));
        DPC_CK(tmp.get(&db.ucount, 4));
        DPC_CK(tmp.get(&db.tree_list, N));
        DPC_CK(tmp.get(&db.bf_list, N));
        DPC_CK(cudaMemsetAsync(db.ucount, 0, 4 * sizeof(uint32_t), st));
        db.tcount = db.ucount;
        db.bf_rank = tune.bf_rank;
        // near pass: a thread per pick while the neighbour cells hold few
        // picks, a warp per pick from 6 picks per cell on average (dense
        // 5.8M x 3: the warp form wins at eps 0.2-0.4, 7-12 picks per cell;
        // the thread form at eps 0.6-1.0, 2-5 picks per cell)
        const bool near_threads = tune.sapprox_near_threads == 2 ? npicks < 6 * std::max<int64_t>(ncells, 1)
                                                                 : tune.sapprox_near_threads != 0;
        DPC_CK(launch_sapprox_first(v, w, sb, db, dim_mask, npicks, npicks, !all_points, near_threads,
                                    st));
        // the pick path's tree leaves hold the cells' picks only: every point
        // that ranks above a pick is a pick (the others have rho 0)
        db.lplist = all_points ? nullptr : sb.plist;
        db.lpstart = all_points ? nullptr : sb.pstart;
        const dpc_status ost = open_points(tmp, "S-Approx-DPC first phase");
        db.lplist = db.lpstart = nullptr;
        DPC_TRY(ost);
        mark(6);
        DPC_CK(keep.get(&rho_pub, N));
        DPC_CK(launch_sapprox_rho_out(v, rho_pub, st));
        unsigned long long sst[2] = {0, 0}, pairs[2] = {0, 0};
        DPC_CK(cudaMemcpyAsync(sst, sb.stats, sizeof(sst), cudaMemcpyDeviceToHost, st));
        DPC_CK(cudaMemcpyAsync(pairs, d_stats, sizeof(pairs), cudaMemcpyDeviceToHost, st));
        DPC_TRY(finish_stats("S-Approx-DPC dependent points"));
        DPC_TRY(settle());  // waits for the copies above too
        sap_pairs = pick_items ? pick_pairs : (int64_t)sst[0];
        nsecond = (int64_t)sst[1];
        cand_pairs = all_points ? (int64_t)(pairs[0] + pairs[1]) : sap_pairs;
        dense_pairs = all_points ? (int64_t)pairs[0] : (pick_items ? pick_pairs : 0);
        ms_rho_dense = all_points ? elapsed(7, 4) : (pick_items ? elapsed(4, 2) : 0.f);
        ms[0] = elapsed(0, 7);
        ms[1] = elapsed(7, 2);
        ms[2] = elapsed(2, 5);
        ms[3] = elapsed(5, 6);
        tmp.release();
        dens.release();
        has_density = true;
        dep_kind = 3;
        return DPC_OK;
    }

    // ------------------------------------------------------------ label
    dpc_status label(const int64_t* rho_min, const int64_t* delta_min) {
        if (dep_kind == 0) DPC_TRY(dependent());  // else the dependent points already held
        if (!v.parent) {
            DPC_CK(keep.get(&v.parent, N));
            DPC_CK(keep.get(&v.label, N));
            DPC_CK(keep.get(&v.ncent, B));
        }
        for (int b = 0; b < B; ++b) {
            hd[b].rho_min = rho_min[b];
            hd[b].delta_min2 = delta_min[b] * delta_min[b];
        }
        DPC_TRY(upload_desc());
        mark(12);
        DPC_CK(launch_labels(v, st));
        mark(13);
        return DPC_OK;
    }

    // Labels of dataset b only (a re-query of one dataset of a batch).
    dpc_status label_one(int b, int64_t rho_min, int64_t delta_min) {
        if (dep_kind == 0) DPC_TRY(dependent());
        if (!v.parent) {
            DPC_CK(keep.get(&v.parent, N));
            DPC_CK(keep.get(&v.label, N));
            DPC_CK(keep.get(&v.ncent, B));
        }
        hd[b].rho_min = rho_min;
        hd[b].delta_min2 = delta_min * delta_min;
        DPC_TRY(upload_desc());
        mark(12);
        DPC_CK(launch_labels_one(v, b, hd[b].pt_off, hd[b].n, st));
        mark(13);
        return DPC_OK;
    }

    // After the batch's jobs are done: later work (re-queries of kept
    // datasets, and the frees) goes to stream s.
    void move_to(cudaStream_t s) {
        st = s;
        keep.st = s;
        dens.st = s;
    }

    dpc_status copy_out(void* dst, const void* src, size_t bytes) {
        if (dst && bytes) DPC_CK(cudaMemcpyAsync(dst, src, bytes, cudaMemcpyDefault, st));
        return DPC_OK;
    }

    std::mutex qmu;  // re-queries of the batch's kept datasets from several threads
};

}  // namespace
}  // namespace dpc

struct dpc_ds {
    std::shared_ptr<dpc::Batch> batch;
    int b = 0;
    dpc_ctx* served = nullptr;  // a kept job's dataset: its device bytes count against this context's cap
    uint64_t held = 0;
};

using dpc::Batch;
using dpc::fail;
using dpc::cuda_fail;

extern "C" {

const char* dpc_last_error(void) { return dpc::g_err.c_str(); }

int64_t dpc_kernel_launches(void) { return (int64_t)dpc::launch_count(); }

dpc_status dpc_create(const dpc_options* opt, dpc_ctx** out) {
    if (!out) return fail(DPC_ERR_INVALID_ARG, "out is NULL");
    *out = nullptr;
    dpc_options o{};
    if (opt) o = *opt;
    int ndev = 0;
    cudaError_t e = cudaGetDeviceCount(&ndev);
    if (e != cudaSuccess) return cuda_fail(e, "cudaGetDeviceCount");
    if (o.device < 0 || o.device >= ndev) return fail(DPC_ERR_INVALID_ARG, "no such device");
    if (o.mode != 0 && o.mode != 1) return fail(DPC_ERR_INVALID_ARG, "mode must be 0 or 1");
    e = cudaSetDevice(o.device);
    if (e != cudaSuccess) return cuda_fail(e, "cudaSetDevice");
    auto* c = new dpc_ctx();
    c->device = o.device;
    c->debug = o.debug_checks;
    c->mode = o.mode;
    c->cap = o.hbm_cap_bytes ? o.hbm_cap_bytes : dpc::kDefaultCap;
    c->max_inflight = o.max_inflight > 0 ? o.max_inflight : 4;
    if (o.tune_cache && o.tune_cache[0]) {
        c->tune_cache = o.tune_cache;
        dpc::load_tune_cache(c);
    }
    if (o.cuda_stream) {
        c->stream = (cudaStream_t)o.cuda_stream;
    } else {
        e = cudaStreamCreateWithFlags(&c->stream, cudaStreamNonBlocking);
        if (e != cudaSuccess) {
            delete c;
            return cuda_fail(e, "cudaStreamCreate");
        }
        c->own_stream = true;
    }
    // keep freed blocks in the device's pool so repeated calls do not go back
    // to the driver
    cudaMemPool_t pool;
    if (cudaDeviceGetDefaultMemPool(&pool, o.device) == cudaSuccess) {
        uint64_t thr = UINT64_MAX;
        cudaMemPoolSetAttribute(pool, cudaMemPoolAttrReleaseThreshold, &thr);
    }
    *out = c;
    return DPC_OK;
}

dpc_status dpc_set_profiling(dpc_ctx* ctx, int on) {
    if (!ctx) return fail(DPC_ERR_INVALID_ARG, "ctx is NULL");
    ctx->profiling = on ? 1 : 0;
    return DPC_OK;
}

dpc_status dpc_set_tuning(dpc_ctx* ctx, const char* key, int64_t value) {
    if (!ctx || !key) return fail(DPC_ERR_INVALID_ARG, "ctx or key is NULL");
    const std::string k(key);
    dpc::Tune& t = ctx->tune;
    if (k == "kch" && value >= 32 && value <= (1 << 20)) t.kch = (int)value;
    else if (k == "qch" && (value == 32 || value == 64 || value == 128)) t.qch = (int)value;
    else if (k == "kmax" && value >= 1 && value <= dpc::kMaxGridDims) t.kmax = (int)value;
    else if (k == "bf_rank" && value >= 0 && value <= UINT32_MAX) t.bf_rank = (uint32_t)value;
    else if (k == "tree_warp" && value >= 0 && value <= 2) t.tree_warp = (int)value;
    else if (k == "hd_cell_factor" && value >= 1 && value <= 3) t.hd_cell_factor = (int)value;
    else if (k == "hd_min_d" && value >= 1 && value <= 9) t.hd_min_d = (int)value;
    else if (k == "sapprox_path" && value >= 0 && value <= 2) t.sapprox_path = (int)value;
    else if (k == "sapprox_ratio" && value >= 1 && value <= 1024) t.sapprox_ratio = (int)value;
    else if (k == "sapprox_rho_cells" && value >= 0 && value <= 3) t.sapprox_rho_cells = (int)value;
    else if (k == "sapprox_near_threads" && value >= 0 && value <= 2) t.sapprox_near_threads = (int)value;
    else if (k == "rho_bulk" && value >= 0 && value <= 1) t.rho_bulk = (int)value;
    else if (k == "sparse_cand" && value >= 0 && value <= (1ll << 31)) t.sparse_cand = (int)std::min<int64_t>(value, INT32_MAX);
    else if (k == "max_batch_jobs" && value >= 1 && value <= 4096) {
        std::lock_guard<std::mutex> lk(ctx->mu);
        ctx->max_batch_jobs = (int)value;
    } else if (k == "max_batch_points" && value >= 1 && value <= (1ll << 31) - 1) {
        std::lock_guard<std::mutex> lk(ctx->mu);
        ctx->max_batch_points = value;
    } else return fail(DPC_ERR_INVALID_ARG, "unknown tuning key or value out of range: " + k);
    return DPC_OK;
}

dpc_status dpc_get_tuning(dpc_ctx* ctx, const char* key, int64_t* value) {
    if (!ctx || !key || !value) return fail(DPC_ERR_INVALID_ARG, "NULL argument");
    const std::string k(key);
    const dpc::Tune& t = ctx->tune;
    if (k == "kch") *value = t.kch;
    else if (k == "qch") *value = t.qch;
    else if (k == "kmax") *value = t.kmax;
    else if (k == "bf_rank") *value = t.bf_rank;
    else if (k == "tree_warp") *value = t.tree_warp;
    else if (k == "hd_cell_factor") *value = t.hd_cell_factor;
    else if (k == "hd_min_d") *value = t.hd_min_d;
    else if (k == "sparse_cand") *value = t.sparse_cand;
    else if (k == "sapprox_path") *value = t.sapprox_path;
    else if (k == "sapprox_ratio") *value = t.sapprox_ratio;
    else if (k == "sapprox_rho_cells") *value = t.sapprox_rho_cells;
    else if (k == "sapprox_near_threads") *value = t.sapprox_near_threads;
    else if (k == "rho_bulk") *value = t.rho_bulk;
    else if (k == "max_batch_jobs") {
        std::lock_guard<std::mutex> lk(ctx->mu);
        *value = ctx->max_batch_jobs;
    } else if (k == "max_batch_points") {
        std::lock_guard<std::mutex> lk(ctx->mu);
        *value = ctx->max_batch_points;
    } else return fail(DPC_ERR_INVALID_ARG, "unknown tuning key: " + k);
    return DPC_OK;
}

static dpc_status check_input(const int32_t* points, int64_t n, int32_t d, int64_t d_cut) {
    if (n < 0 || n >= (1ll << 31)) return fail(DPC_ERR_INVALID_ARG, "n must be in [0, 2^31)");
    if (d < 1 || d > 8) return fail(DPC_ERR_INVALID_ARG, "d must be in [1, 8]");
    if (d_cut < 1 || d_cut >= (1ll << 31)) return fail(DPC_ERR_INVALID_ARG, "d_cut must be in [1, 2^31)");
    if (n > 0 && !points) return fail(DPC_ERR_INVALID_ARG, "points is NULL");
    return DPC_OK;
}

dpc_status dpc_density(dpc_ctx* ctx, const int32_t* points, int64_t n, int32_t d, int64_t d_cut, int is_device,
                       dpc_ds** out, int32_t* rho_out) {
    if (!ctx || !out) return fail(DPC_ERR_INVALID_ARG, "ctx or out is NULL");
    *out = nullptr;
    DPC_TRY(check_input(points, n, d, d_cut));
    cudaError_t e = cudaSetDevice(ctx->device);
    if (e != cudaSuccess) return cuda_fail(e, "cudaSetDevice");
    auto b = std::make_shared<Batch>();
    b->ctx = ctx;
    std::vector<dpc::Input> in{{points, n, d, d_cut, is_device}};
    DPC_TRY(b->density(in));
    if (rho_out) DPC_TRY(b->copy_out(rho_out, b->v.rho, sizeof(int32_t) * n));
    DPC_TRY(b->settle());  // the statistics, the error word, and the copy done
    auto* ds = new dpc_ds();
    ds->batch = b;
    ds->b = 0;
    b->refs = 1;
    *out = ds;
    return DPC_OK;
}

dpc_status dpc_sapprox(dpc_ctx* ctx, const int32_t* points, int64_t n, int32_t d, int64_t d_cut, int64_t eps_num,
                       int64_t eps_den, int is_device, dpc_ds** out, int32_t* rho_out, int32_t* dep_out,
                       int64_t* delta2_out, uint8_t* pick_out) {
    if (!ctx || !out) return fail(DPC_ERR_INVALID_ARG, "ctx or out is NULL");
    *out = nullptr;
    DPC_TRY(check_input(points, n, d, d_cut));
    if (eps_num < 1 || eps_num > (1 << 20) || eps_den < 1 || eps_den > (1 << 20))
        return fail(DPC_ERR_INVALID_ARG, "eps_num and eps_den must be in [1, 2^20]");
    cudaError_t e = cudaSetDevice(ctx->device);
    if (e != cudaSuccess) return cuda_fail(e, "cudaSetDevice");
    auto b = std::make_shared<Batch>();
    b->ctx = ctx;
    std::vector<dpc::Input> in{{points, n, d, d_cut, is_device}};
    DPC_TRY(b->sapprox(in, {eps_num}, {eps_den}));
    DPC_TRY(b->copy_out(rho_out, b->rho_pub, sizeof(int32_t) * n));
    DPC_TRY(b->copy_out(dep_out, b->v.dep, sizeof(int32_t) * n));
    DPC_TRY(b->copy_out(delta2_out, b->v.delta2, sizeof(int64_t) * n));
    DPC_TRY(b->copy_out(pick_out, b->v.pick, sizeof(uint8_t) * n));
    DPC_TRY(b->sync("copy S-Approx-DPC results"));
    auto* ds = new dpc_ds();
    ds->batch = b;
    ds->b = 0;
    b->refs = 1;
    *out = ds;
    return DPC_OK;
}

dpc_status dpc_cluster(dpc_ctx* ctx, const int32_t* points, int64_t n, int32_t d, int64_t d_cut, int is_device,
                       int64_t rho_min, int64_t delta_min, int32_t* rho_out, int32_t* dep_out, int64_t* delta2_out,
                       int32_t* label_out, int64_t* n_centers) {
    if (!ctx) return fail(DPC_ERR_INVALID_ARG, "ctx is NULL");
    DPC_TRY(check_input(points, n, d, d_cut));
    if (delta_min <= d_cut || delta_min > dpc::kMaxDeltaMin)
        return fail(DPC_ERR_INVALID_ARG, "delta_min must be in (d_cut, 3037000499]");
    cudaError_t e = cudaSetDevice(ctx->device);
    if (e != cudaSuccess) return cuda_fail(e, "cudaSetDevice");
    {
        std::lock_guard<std::mutex> lk(ctx->mu);
        if (!ctx->copy_stream) {
            for (auto& ev : ctx->copy_ev)
                if ((e = cudaEventCreateWithFlags(&ev, cudaEventDisableTiming)) != cudaSuccess)
                    return cuda_fail(e, "cudaEventCreate");
            if ((e = cudaStreamCreateWithFlags(&ctx->copy_stream, cudaStreamNonBlocking)) != cudaSuccess)
                return cuda_fail(e, "cudaStreamCreate");
        }
    }
    Batch bt;
    bt.ctx = ctx;
    // on every way out, the side copies end before the batch frees its buffers
    struct CopyWait {
        cudaStream_t s;
        ~CopyWait() { cudaStreamSynchronize(s); }
    } copy_wait{ctx->copy_stream};
    std::vector<dpc::Input> in{{points, n, d, d_cut, is_device}};
    DPC_TRY(bt.density(in));
    cudaStream_t cs = ctx->copy_stream;
    auto side_copy = [&](void* dst, const void* src, size_t bytes) -> dpc_status {
        if (dst && bytes) DPC_CK(cudaMemcpyAsync(dst, src, bytes, cudaMemcpyDefault, cs));
        return DPC_OK;
    };
    // rho is final: it travels while the dependent points are computed
    DPC_CK(cudaEventRecord(ctx->copy_ev[0], bt.st));
    DPC_CK(cudaStreamWaitEvent(cs, ctx->copy_ev[0], 0));
    DPC_TRY(side_copy(rho_out, bt.v.rho, sizeof(int32_t) * n));
    DPC_TRY(bt.dependent());
    // the dependent points travel while the labels are computed
    DPC_CK(cudaEventRecord(ctx->copy_ev[1], bt.st));
    DPC_CK(cudaStreamWaitEvent(cs, ctx->copy_ev[1], 0));
    DPC_TRY(side_copy(dep_out, bt.v.dep, sizeof(int32_t) * n));
    DPC_TRY(side_copy(delta2_out, bt.v.delta2, sizeof(int64_t) * n));
    DPC_TRY(bt.label(&rho_min, &delta_min));
    DPC_TRY(bt.copy_out(label_out, bt.v.label, sizeof(int32_t) * n));
    unsigned long long nc = 0;
    if (n_centers) DPC_TRY(bt.copy_out(&nc, bt.v.ncent, sizeof(nc)));
    DPC_TRY(bt.sync("labels"));
    e = cudaStreamSynchronize(cs);
    if (e != cudaSuccess) return cuda_fail(e, "copies");
    DPC_TRY(bt.settle());
    DPC_TRY(bt.check_err("labels"));
    if (n_centers) *n_centers = (int64_t)nc;
    return DPC_OK;
}

dpc_status dpc_dependent(dpc_ds* ds, int32_t* dep_out, int64_t* delta2_out) {
    if (!ds || !ds->batch) return fail(DPC_ERR_STATE, "invalid dataset handle");
    Batch& bt = *ds->batch;
    cudaSetDevice(bt.ctx->device);
    DPC_TRY(bt.dependent());
    const dpc::DsDesc& h = bt.hd[ds->b];
    DPC_TRY(bt.copy_out(dep_out, bt.v.dep + h.pt_off, sizeof(int32_t) * h.n));
    DPC_TRY(bt.copy_out(delta2_out, bt.v.delta2 + h.pt_off, sizeof(int64_t) * h.n));
    DPC_TRY(bt.sync("copy dependent"));
    return bt.settle();
}

dpc_status dpc_dependent_approx(dpc_ds* ds, int32_t* dep_out, int64_t* delta2_out, uint8_t* exact_out) {
    if (!ds || !ds->batch) return fail(DPC_ERR_STATE, "invalid dataset handle");
    Batch& bt = *ds->batch;
    cudaSetDevice(bt.ctx->device);
    DPC_TRY(bt.dependent_approx());
    const dpc::DsDesc& h = bt.hd[ds->b];
    DPC_TRY(bt.copy_out(dep_out, bt.v.dep + h.pt_off, sizeof(int32_t) * h.n));
    DPC_TRY(bt.copy_out(delta2_out, bt.v.delta2 + h.pt_off, sizeof(int64_t) * h.n));
    DPC_TRY(bt.copy_out(exact_out, bt.v.exact + h.pt_off, sizeof(uint8_t) * h.n));
    DPC_TRY(bt.sync("copy approximate dependent"));
    return bt.settle();
}

dpc_status dpc_label(dpc_ds* ds, int64_t rho_min, int64_t delta_min, int32_t* label_out, int64_t* n_centers) {
    if (!ds || !ds->batch) return fail(DPC_ERR_STATE, "invalid dataset handle");
    Batch& bt = *ds->batch;
    const dpc::DsDesc& h = bt.hd[ds->b];
    if (delta_min <= h.d_cut || delta_min > dpc::kMaxDeltaMin)
        return fail(DPC_ERR_INVALID_ARG, "delta_min must be in (d_cut, 3037000499]");
    cudaSetDevice(bt.ctx->device);
    std::lock_guard<std::mutex> lk(bt.qmu);
    DPC_TRY(bt.label_one(ds->b, rho_min, delta_min));
    DPC_TRY(bt.copy_out(label_out, bt.v.label + h.pt_off, sizeof(int32_t) * h.n));
    unsigned long long nc = 0;
    if (n_centers) DPC_TRY(bt.copy_out(&nc, bt.v.ncent + ds->b, sizeof(nc)));
    DPC_TRY(bt.sync("labels"));
    DPC_TRY(bt.settle());
    DPC_TRY(bt.check_err("labels"));
    bt.ms[5] = bt.elapsed(12, 13);
    if (n_centers) *n_centers = (int64_t)nc;
    return DPC_OK;
}

dpc_status dpc_release(dpc_ds* ds) {
    if (!ds) return fail(DPC_ERR_STATE, "invalid dataset handle");
    if (ds->batch) {
        cudaSetDevice(ds->batch->ctx->device);
        cudaStreamSynchronize(ds->batch->st);
    }
    dpc_ctx* ctx = ds->served;
    const uint64_t held = ds->held;
    delete ds;  // the batch's memory goes with its last dataset
    if (ctx) {
        std::lock_guard<std::mutex> lk(ctx->mu);
        ctx->held_bytes -= held;
        ctx->cv.notify_all();
    }
    return DPC_OK;
}

static void fill_info(const Batch& bt, int b, dpc_info* out) {
    std::memset(out, 0, sizeof(*out));
    const dpc::DsDesc& h = bt.hd[b];
    out->n = h.n;
    out->cells = bt.ncells;
    out->dense_cells = bt.ndense;
    out->work_items = bt.nitems;
    out->open_after_ring = bt.ntree + bt.nbf;
    out->brute_points = bt.nbf;
    out->grid_dims = h.k;
    out->pair_bits = h.w32 ? 32 : 64;
    out->ms_grid = bt.ms[0];
    out->ms_rho = bt.ms[1];
    out->ms_rank = bt.ms[2];
    out->ms_ring = bt.ms[3];
    out->ms_rest = bt.ms[4];
    out->ms_label = bt.ms[5];
    out->cand_pairs = bt.cand_pairs;
    out->tree_visits = bt.tree_visits;
    out->tree_pairs = bt.tree_pairs;
    out->pair_mode = h.mode;
    out->dense_pairs = bt.dense_pairs;
    out->ms_rho_dense = bt.ms_rho_dense;
    out->grid_key_bits = bt.grid_key_bits;
    out->rank_key_bits = bt.rank_key_bits;
    out->picks = bt.npicks;
    out->second_phase = bt.nsecond;
    out->density_path = bt.density_path;
    out->device_bytes_peak = (int64_t)bt.meter.peak;
}

dpc_status dpc_ds_info(const dpc_ds* ds, dpc_info* out) {
    if (!ds || !ds->batch || !out) return fail(DPC_ERR_INVALID_ARG, "NULL argument");
    {
        std::lock_guard<std::mutex> lk(ds->batch->qmu);
        cudaSetDevice(ds->batch->ctx->device);
        DPC_TRY(ds->batch->settle());
    }
    fill_info(*ds->batch, ds->b, out);
    return DPC_OK;
}

dpc_status dpc_last_batch_info(dpc_ctx* ctx, dpc_info* out) {
    if (!ctx || !out) return fail(DPC_ERR_INVALID_ARG, "NULL argument");
    std::lock_guard<std::mutex> lk(ctx->mu);
    if (!ctx->has_last) return fail(DPC_ERR_STATE, "no batch of jobs has finished on this context");
    *out = ctx->last_info;
    return DPC_OK;
}

}  // extern "C"

// ------------------------------------------------------------------ jobs

namespace dpc {
namespace {

using JobPtr = std::shared_ptr<dpc_ctx::JobRec>;

// Device bytes one job holds at its peak: per point a base for the records,
// the per-point state, the sort buffers and the cell tree, 8 bytes per
// dimension, one 8-byte run slot per neighbour cell of the grid (a cell keeps
// (2R+1)^k slots, and there is at most one cell per point), and the second
// grid of the approximate methods; plus 16 MB. Measured peaks of the served
// trace's problems lie below it: 180-290 bytes per point in 2-3 dims,
// 390-680 in 4-6 (81 slots), 2.7-4.3 KB in 7-8 (625 slots, cell factor 2),
// and up to 465 (S-Approx-DPC) in 3 dims.
uint64_t job_bytes(int64_t n, int32_t d, int32_t method, const Tune& t) {
    const int k = std::min(std::min<int>(d, t.kmax), kMaxGridDims);
    const int R = d >= t.hd_min_d ? t.hd_cell_factor : 1;
    uint64_t slots = 1;
    for (int j = 0; j < k; ++j) slots *= (uint64_t)(2 * R + 1);
    const uint64_t per = 176 + 8 * (uint64_t)d + 8 * slots + (method == 1 ? 96 : (method == 2 ? 160 : 0));
    return (uint64_t)n * per + (16ull << 20);
}

}  // namespace
}  // namespace dpc

extern "C" uint64_t dpc_job_footprint(dpc_ctx* ctx, int64_t n, int32_t d, int32_t method) {
    const dpc::Tune t = ctx ? ctx->tune : dpc::Tune{};
    return dpc::job_bytes(n < 0 ? 0 : n, d < 1 ? 1 : (d > 8 ? 8 : d), method, t);
}

namespace dpc {
namespace {

// One job's outputs are written: its status, for dpc_poll and dpc_wait.
void mark_done(dpc_ctx* ctx, const JobPtr& j, dpc_status s) {
    std::lock_guard<std::mutex> lk(ctx->mu);
    if (j->status != DPC_PENDING) return;
    j->status = s;
    j->t_done = std::chrono::steady_clock::now();
    ctx->cv.notify_all();
}

// Run a group of jobs as one batch on stream st; fills their outputs. Each
// job is marked done as soon as its own outputs are written.
dpc_status run_jobs(dpc_ctx* ctx, std::vector<JobPtr>& jobs, cudaStream_t st) {
    auto bt = std::make_shared<Batch>();
    bt->ctx = ctx;
    bt->st = st;
    std::vector<Input> in;
    int maxq = 0;
    for (auto& j : jobs) {
        in.push_back({j->job.points, j->job.n, j->job.d, j->job.d_cut, j->job.is_device ? 1 : 0});
        maxq = std::max(maxq, j->job.n_queries);
    }
    // one method per batch (the callers group the jobs)
    const int method = jobs.empty() ? 0 : jobs[0]->job.method;
    if (method == 2) {
        std::vector<int64_t> en, ed;
        for (auto& j : jobs) {
            en.push_back(j->job.eps_num);
            ed.push_back(j->job.eps_den);
        }
        DPC_TRY(bt->sapprox(in, en, ed));
    } else {
        DPC_TRY(bt->density(in));
        if (method == 1) DPC_TRY(bt->dependent_approx());
        else DPC_TRY(bt->dependent());
    }
    // outputs: those the device can write (device memory; in a batch of
    // several jobs, page-locked host memory too) in one kernel pass per kind,
    // the others by one copy per array
    const int32_t* rho_src = method == 2 ? bt->rho_pub : bt->v.rho;
    const uint8_t* aux_src = method == 2 ? bt->v.pick : (method == 1 ? bt->v.exact : nullptr);
    std::vector<OutJob> oj;
    std::vector<char> by_kernel(jobs.size(), 0);
    int64_t dtot = 0;
    for (size_t b = 0; b < jobs.size(); ++b) {
        const dpc_job& jb = jobs[b]->job;
        const DsDesc& h = bt->hd[b];
        OutJob o{};
        bool kern = jb.is_device != 0;
        if (kern) {
            o.rho = jb.rho_out;
            o.dep = jb.dep_out;
            o.delta2 = jb.delta2_out;
            o.aux = method != 0 ? jb.aux_out : nullptr;
            o.label = jb.label_out;
        } else if (jobs.size() > 1) {
            kern = true;
            auto view = [&kern](auto* p) {
                using T = std::remove_pointer_t<decltype(p)>;
                T* d = static_cast<T*>(device_view(p));
                kern = kern && (p == nullptr || d != nullptr);
                return d;
            };
            o.rho = view(jb.rho_out);
            o.dep = view(jb.dep_out);
            o.delta2 = view(jb.delta2_out);
            o.aux = method != 0 ? view(jb.aux_out) : nullptr;
            o.label = view(jb.label_out);
        }
        if (kern) {
            by_kernel[b] = 1;
            if (h.n == 0) continue;
            o.src_off = h.pt_off;
            o.dst_off = dtot;
            o.n = h.n;
            o.nq = jb.n_queries;
            oj.push_back(o);
            dtot += h.n;
            continue;
        }
        DPC_TRY(bt->copy_out(jb.rho_out, rho_src + h.pt_off, sizeof(int32_t) * h.n));
        DPC_TRY(bt->copy_out(jb.dep_out, bt->v.dep + h.pt_off, sizeof(int32_t) * h.n));
        DPC_TRY(bt->copy_out(jb.delta2_out, bt->v.delta2 + h.pt_off, sizeof(int64_t) * h.n));
        if (method != 0) DPC_TRY(bt->copy_out(jb.aux_out, aux_src + h.pt_off, h.n));
    }
    OutJob* d_oj = nullptr;
    if (!oj.empty()) {
        DPC_CK(bt->keep.get(&d_oj, oj.size()));
        DPC_CK(cudaMemcpyAsync(d_oj, oj.data(), sizeof(OutJob) * oj.size(), cudaMemcpyHostToDevice, st));
        DPC_CK(launch_job_outputs(d_oj, (int)oj.size(), dtot, rho_src, bt->v.dep, bt->v.delta2, aux_src, nullptr, 0,
                                  0, st));
    }
    std::vector<int64_t> rmin(jobs.size()), dmin(jobs.size());
    std::vector<unsigned long long> nc(jobs.size());
    for (int q = 0; q < maxq; ++q) {
        for (size_t b = 0; b < jobs.size(); ++b) {
            const int qq = std::min(q, jobs[b]->job.n_queries - 1);
            rmin[b] = jobs[b]->rmin[qq];
            dmin[b] = jobs[b]->dmin[qq];
        }
        DPC_TRY(bt->label(rmin.data(), dmin.data()));
        DPC_TRY(bt->copy_out(nc.data(), bt->v.ncent, sizeof(unsigned long long) * jobs.size()));
        if (d_oj)
            DPC_CK(launch_job_outputs(d_oj, (int)oj.size(), dtot, nullptr, nullptr, nullptr, nullptr, bt->v.label, 1, q,
                                      bt->st));
        for (size_t b = 0; b < jobs.size(); ++b) {
            const dpc_job& jb = jobs[b]->job;
            if (by_kernel[b] || q >= jb.n_queries || !jb.label_out) continue;
            const DsDesc& h = bt->hd[b];
            DPC_TRY(bt->copy_out(jb.label_out + (int64_t)q * h.n, bt->v.label + h.pt_off, sizeof(int32_t) * h.n));
        }
        DPC_TRY(bt->sync("labels"));
        DPC_TRY(bt->check_err("labels"));
        for (size_t b = 0; b < jobs.size(); ++b)
            if (q < jobs[b]->job.n_queries && jobs[b]->job.n_centers_out)
                jobs[b]->job.n_centers_out[q] = (int64_t)nc[b];
        // every job whose last query this was is done: its outputs are
        // written (a kept job once the batch is no longer in use here)
        for (size_t b = 0; b < jobs.size(); ++b)
            if (jobs[b]->job.n_queries == q + 1 && !jobs[b]->job.keep) mark_done(ctx, jobs[b], DPC_OK);
    }
    // kept datasets: re-queries (and the frees) run on the context's stream
    bool any_kept = false;
    for (auto& j : jobs) any_kept |= j->job.keep != 0;
    if (any_kept) {
        bt->move_to(ctx->stream);
        for (size_t b = 0; b < jobs.size(); ++b) {
            if (!jobs[b]->job.keep) continue;
            jobs[b]->kept = bt;
            jobs[b]->kept_b = (int)b;
            mark_done(ctx, jobs[b], DPC_OK);
        }
    }
    // the batch's counters and stage times (the first dataset's per-dataset
    // fields, the batch's totals)
    DPC_TRY(bt->settle());
    dpc_info info;
    fill_info(*bt, 0, &info);
    int64_t n = 0;
    for (auto& j : jobs) n += j->job.n;
    info.n = n;
    std::lock_guard<std::mutex> lk(ctx->mu);
    ctx->last_info = info;
    ctx->has_last = true;
    return DPC_OK;
}

// The batch is over: jobs not yet done get its status (an error), and the
// device bytes of every job not kept are released (a kept job's bytes stay
// held until its dataset is released).
void finish(dpc_ctx* ctx, std::vector<JobPtr>& group, dpc_status s) {
    std::lock_guard<std::mutex> lk(ctx->mu);
    const auto now = std::chrono::steady_clock::now();
    for (auto& j : group) {
        if (j->status == DPC_PENDING) {
            j->status = s == DPC_OK ? DPC_ERR_STATE : s;
            j->t_done = now;
        }
        if (j->status != DPC_OK) j->kept.reset();
        // a kept job's bytes are released with its dataset (or by the result
        // call that frees it), never here
        if (!(j->status == DPC_OK && j->job.keep)) ctx->held_bytes -= j->bytes;
    }
    ctx->cv.notify_all();
}

// Served mode: each worker owns a stream and admits the jobs waiting at the
// head of the queue while they fit the memory cap, runs them as one batch,
// and goes back for more. With several workers, a batch is admitted and
// launched while earlier batches are still running on the device.
void serve_loop(dpc_ctx* ctx) {
    cudaSetDevice(ctx->device);
    cudaStream_t st = nullptr;
    cudaStreamCreateWithFlags(&st, cudaStreamNonBlocking);
    while (true) {
        std::vector<JobPtr> group;
        {
            std::unique_lock<std::mutex> lk(ctx->mu);
            ctx->cv.wait(lk, [&] {
                if (ctx->stop) return true;
                if (ctx->waiting.empty()) return false;
                auto it = ctx->jobs.find(ctx->waiting.front());
                return it == ctx->jobs.end() || ctx->held_bytes + it->second->bytes <= ctx->cap;
            });
            if (ctx->stop && ctx->waiting.empty()) break;
            // the points cap keeps a small job out of a large job's batch; with
            // a backlog every worker's share of it may go in one batch instead
            // (larger batches, fewer fixed costs, while all of them wait anyway)
            int64_t backlog = 0;
            for (uint64_t t : ctx->waiting) {
                auto jt = ctx->jobs.find(t);
                if (jt != ctx->jobs.end()) backlog += jt->second->job.n;
            }
            const int64_t cap_points =
                std::max<int64_t>(ctx->max_batch_points, backlog / std::max(1, ctx->max_inflight));
            int64_t pts = 0;
            while (!ctx->waiting.empty() && (int)group.size() < ctx->max_batch_jobs) {
                auto it = ctx->jobs.find(ctx->waiting.front());
                if (it == ctx->jobs.end()) {
                    ctx->waiting.pop_front();
                    continue;
                }
                JobPtr j = it->second;
                if (ctx->held_bytes + j->bytes > ctx->cap) break;
                if (!group.empty() && j->job.method != group[0]->job.method) break;  // one method per batch
                if (pts + j->job.n >= (1ll << 31) - 1) break;
                if (!group.empty() && pts + j->job.n > cap_points) break;  // a large job runs alone
                ctx->waiting.pop_front();
                ctx->held_bytes += j->bytes;
                pts += j->job.n;
                j->t_admit = std::chrono::steady_clock::now();
                group.push_back(j);
            }
        }
        if (group.empty()) continue;
        dpc_status s = run_jobs(ctx, group, st);
        finish(ctx, group, s);
    }
    cudaStreamDestroy(st);
}

dpc_status check_job(const dpc_job* j) {
    if (!j) return fail(DPC_ERR_INVALID_ARG, "job is NULL");
    if (j->n < 0 || j->n >= (1ll << 31)) return fail(DPC_ERR_INVALID_ARG, "n must be in [0, 2^31)");
    if (j->d < 1 || j->d > 8) return fail(DPC_ERR_INVALID_ARG, "d must be in [1, 8]");
    if (j->d_cut < 1 || j->d_cut >= (1ll << 31)) return fail(DPC_ERR_INVALID_ARG, "d_cut must be in [1, 2^31)");
    if (j->n > 0 && !j->points) return fail(DPC_ERR_INVALID_ARG, "points is NULL");
    if (j->is_device != 0 && j->is_device != 1) return fail(DPC_ERR_INVALID_ARG, "is_device must be 0 or 1");
    if (j->n_queries < 1 || !j->rho_min || !j->delta_min)
        return fail(DPC_ERR_INVALID_ARG, "a job needs at least one (rho_min, delta_min) query");
    for (int q = 0; q < j->n_queries; ++q)
        if (j->delta_min[q] <= j->d_cut || j->delta_min[q] > kMaxDeltaMin)
            return fail(DPC_ERR_INVALID_ARG, "delta_min must be in (d_cut, 3037000499]");
    if (j->method < 0 || j->method > 2) return fail(DPC_ERR_INVALID_ARG, "method must be 0, 1 or 2");
    if (j->method == 2 && (j->eps_num < 1 || j->eps_num > (1 << 20) || j->eps_den < 1 || j->eps_den > (1 << 20)))
        return fail(DPC_ERR_INVALID_ARG, "eps_num and eps_den must be in [1, 2^20]");
    return DPC_OK;
}

}  // namespace
}  // namespace dpc

extern "C" {

dpc_status dpc_submit(dpc_ctx* ctx, const dpc_job* job, uint64_t* ticket) {
    if (!ctx || !ticket) return fail(DPC_ERR_INVALID_ARG, "ctx or ticket is NULL");
    DPC_TRY(dpc::check_job(job));
    auto rec = std::make_shared<dpc_ctx::JobRec>();
    rec->job = *job;
    rec->rmin.assign(job->rho_min, job->rho_min + job->n_queries);
    rec->dmin.assign(job->delta_min, job->delta_min + job->n_queries);
    rec->bytes = dpc::job_bytes(job->n, job->d, job->method, ctx->tune);
    rec->t_submit = std::chrono::steady_clock::now();
    if (ctx->mode == 1 && rec->bytes > ctx->cap) return fail(DPC_ERR_CAPACITY, "job exceeds the memory cap");
    std::lock_guard<std::mutex> lk(ctx->mu);
    if (ctx->mode == 1 && ctx->workers.empty()) {
        for (int i = 0; i < ctx->max_inflight; ++i) ctx->workers.emplace_back(dpc::serve_loop, ctx);
    }
    const uint64_t t = ctx->next_ticket++;
    ctx->jobs[t] = rec;
    ctx->waiting.push_back(t);
    *ticket = t;
    ctx->cv.notify_all();
    return DPC_OK;
}

// The result of a finished job (ctx->mu held). A kept job's dataset is
// handed out here, once; with out NULL it is freed instead.
static void fill_result(dpc_ctx* ctx, dpc_ctx::JobRec& j, dpc_result* out) {
    dpc_ds* ds = nullptr;
    if (j.kept) {
        if (out) {
            ds = new dpc_ds;
            ds->batch = std::move(j.kept);
            ds->b = j.kept_b;
            ds->served = ctx;
            ds->held = j.bytes;
        } else {
            ctx->held_bytes -= j.bytes;
            ctx->cv.notify_all();
        }
        j.kept.reset();
    }
    if (!out) return;
    out->status = j.status;
    out->queue_ms = std::chrono::duration<double, std::milli>(j.t_admit - j.t_submit).count();
    out->run_ms = std::chrono::duration<double, std::milli>(j.t_done - j.t_admit).count();
    out->dataset = ds;
}

dpc_status dpc_poll(dpc_ctx* ctx, uint64_t ticket, dpc_result* out) {
    if (!ctx) return fail(DPC_ERR_INVALID_ARG, "ctx is NULL");
    std::lock_guard<std::mutex> lk(ctx->mu);
    auto it = ctx->jobs.find(ticket);
    if (it == ctx->jobs.end()) return fail(DPC_ERR_STATE, "unknown ticket");
    if (it->second->status == DPC_PENDING) {
        if (out) out->status = DPC_PENDING;
        return DPC_PENDING;
    }
    fill_result(ctx, *it->second, out);
    const dpc_status s = it->second->status;
    ctx->jobs.erase(it);
    return s;
}

dpc_status dpc_wait(dpc_ctx* ctx, uint64_t ticket, int64_t timeout_ms, dpc_result* out) {
    if (!ctx) return fail(DPC_ERR_INVALID_ARG, "ctx is NULL");
    std::unique_lock<std::mutex> lk(ctx->mu);
    auto it = ctx->jobs.find(ticket);
    if (it == ctx->jobs.end()) return fail(DPC_ERR_STATE, "unknown ticket");
    auto rec = it->second;
    const bool done = ctx->cv.wait_for(lk, std::chrono::milliseconds(timeout_ms < 0 ? 0 : timeout_ms),
                                       [&] { return rec->status != DPC_PENDING; });
    if (!done) return fail(DPC_ERR_TIMEOUT, "job not finished within the timeout");
    fill_result(ctx, *rec, out);
    ctx->jobs.erase(ticket);
    return rec->status;
}

dpc_status dpc_flush(dpc_ctx* ctx) {
    if (!ctx) return fail(DPC_ERR_INVALID_ARG, "ctx is NULL");
    if (ctx->mode != 0) return fail(DPC_ERR_STATE, "dpc_flush is for batched mode");
    std::vector<dpc::JobPtr> group;
    {
        std::lock_guard<std::mutex> lk(ctx->mu);
        const auto now = std::chrono::steady_clock::now();
        while (!ctx->waiting.empty()) {
            auto it = ctx->jobs.find(ctx->waiting.front());
            ctx->waiting.pop_front();
            if (it == ctx->jobs.end()) continue;
            it->second->t_admit = now;
            ctx->held_bytes += it->second->bytes;
            group.push_back(it->second);
        }
    }
    if (group.empty()) return DPC_OK;
    cudaSetDevice(ctx->device);
    // consecutive runs of one method, each one batch
    dpc_status first_err = DPC_OK;
    for (size_t a = 0; a < group.size();) {
        size_t e = a + 1;
        while (e < group.size() && group[e]->job.method == group[a]->job.method) ++e;
        std::vector<dpc::JobPtr> part(group.begin() + a, group.begin() + e);
        const dpc_status s = dpc::run_jobs(ctx, part, ctx->stream);
        dpc::finish(ctx, part, s);
        if (s != DPC_OK && first_err == DPC_OK) first_err = s;
        a = e;
    }
    return first_err;
}

dpc_status dpc_autotune(dpc_ctx* ctx, const dpc_job* jobs, int32_t n_jobs, int32_t repeats, char* report,
                        size_t report_len) {
    if (!ctx || !jobs || n_jobs < 1) return fail(DPC_ERR_INVALID_ARG, "ctx or jobs is NULL, or n_jobs < 1");
    if (repeats < 1 || repeats > 100) return fail(DPC_ERR_INVALID_ARG, "repeats must be in [1, 100]");
    std::vector<dpc::JobPtr> group;
    std::vector<dpc::Input> in;
    for (int i = 0; i < n_jobs; ++i) {
        DPC_TRY(dpc::check_job(&jobs[i]));
        auto rec = std::make_shared<dpc_ctx::JobRec>();
        rec->job = jobs[i];
        rec->rmin.assign(jobs[i].rho_min, jobs[i].rho_min + jobs[i].n_queries);
        rec->dmin.assign(jobs[i].delta_min, jobs[i].delta_min + jobs[i].n_queries);
        group.push_back(rec);
        in.push_back({jobs[i].points, jobs[i].n, jobs[i].d, jobs[i].d_cut, jobs[i].is_device ? 1 : 0});
    }
    const auto sig = dpc::tune_signature(in);
    cudaSetDevice(ctx->device);
    dpc::Tune best;
    {
        std::lock_guard<std::mutex> lk(ctx->mu);
        best = ctx->tune;
    }
    dpc_status err = DPC_OK;
    // best of `repeats` synchronous runs of the sample under knobs t
    auto time_with = [&](const dpc::Tune& t) {
        {
            std::lock_guard<std::mutex> lk(ctx->mu);
            ctx->tuned[sig] = t;
        }
        double ms = 1e300;
        for (int r = 0; r < repeats && err == DPC_OK; ++r) {
            const auto t0 = std::chrono::steady_clock::now();
            err = dpc::run_jobs(ctx, group, ctx->stream);
            const auto t1 = std::chrono::steady_clock::now();
            ms = std::min(ms, std::chrono::duration<double, std::milli>(t1 - t0).count());
        }
        return ms;
    };
    // coordinate descent over the knobs that change speed only
    double cur = time_with(best);
    struct Knob {
        const char* name;
        std::vector<int64_t> values;
    };
    // kch, qch: candidates and queries per dense work item (queries per item
    // set the warps per cell); hd_min_d with the cell factor: cells of side
    // d_cut / f from that many dims up (2: every dataset, the low-d cell factor)
    std::vector<Knob> knobs = {{"kch", {1024, 2048, 4096}}, {"qch", {128, 64, 32}},
                               {"bf_rank", {256, 1024, 4096}}, {"hd_min_d", {7, 2}}};
    if (sig.first >= 4) knobs.push_back({"kmax", {3, 4}});
    knobs.push_back({"hd_cell_factor", {1, 2}});
    auto with = [](dpc::Tune t, const std::string& k, int64_t v) {
        if (k == "kch") t.kch = (int)v;
        else if (k == "qch") t.qch = (int)v;
        else if (k == "hd_min_d") t.hd_min_d = (int)v;
        else if (k == "bf_rank") t.bf_rank = (uint32_t)v;
        else if (k == "kmax") t.kmax = (int)v;
        else if (k == "hd_cell_factor") t.hd_cell_factor = (int)v;
        return t;
    };
    for (const auto& k : knobs) {
        for (int64_t v : k.values) {
            if (err != DPC_OK) break;
            const dpc::Tune t = with(best, k.name, v);
            if (dpc::tune_line(sig, t) == dpc::tune_line(sig, best)) continue;
            const double ms = time_with(t);
            if (err == DPC_OK && ms < 0.98 * cur) {  // keep a change only when it is clearly faster
                best = t;
                cur = ms;
            }
        }
    }
    {
        std::lock_guard<std::mutex> lk(ctx->mu);
        ctx->tuned[sig] = best;
        ctx->tune = best;
    }
    if (err != DPC_OK) return err;
    if (!ctx->tune_cache.empty()) {
        std::lock_guard<std::mutex> lk(ctx->mu);
        if (!dpc::save_tune_cache(ctx)) return fail(DPC_ERR_STATE, "cannot write the tune cache " + ctx->tune_cache);
    }
    if (report && report_len > 0) {
        std::ostringstream o;
        o << dpc::tune_line(sig, best) << " ms=" << cur;
        const std::string r = o.str();
        const size_t m = std::min(report_len - 1, r.size());
        std::memcpy(report, r.data(), m);
        report[m] = '\0';
    }
    return DPC_OK;
}

dpc_status dpc_destroy(dpc_ctx* ctx) {
    if (!ctx) return fail(DPC_ERR_INVALID_ARG, "ctx is NULL");
    {
        std::lock_guard<std::mutex> lk(ctx->mu);
        ctx->stop = true;
        ctx->cv.notify_all();
    }
    for (auto& t : ctx->workers) t.join();
    cudaSetDevice(ctx->device);
    // kept datasets of jobs never collected: freed while their stream lives
    ctx->jobs.clear();
    cudaStreamSynchronize(ctx->stream);
    if (ctx->copy_stream) {
        cudaStreamSynchronize(ctx->copy_stream);
        cudaStreamDestroy(ctx->copy_stream);
    }
    for (auto& e : ctx->copy_ev)
        if (e) cudaEventDestroy(e);
    if (ctx->own_stream) cudaStreamDestroy(ctx->stream);
    delete ctx;
    return DPC_OK;
}

}  // extern "C"
