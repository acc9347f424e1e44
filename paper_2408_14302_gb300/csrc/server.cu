// Continuous-batching server over libcwth plans (host code; no paper
// counterpart: the paper transforms one clip at a time).
//
// Requests wait in arrival order.  A poll first retires the batches whose
// completion event has fired, then fills free stream slots: the oldest
// waiting request and later ones of the same (sample rate, scale count,
// hop, power-of-two length bucket) form a batch of up to max_batch clips.
// The admission budget charges the staging of every batch in flight plus
// the device bytes of every cached plan; the plan cache evicts the least
// recently used idle plan when a new one would exceed its own bound.  Each
// request's samples are read from the caller's memory (in place by a
// gather kernel when page-locked) and its scalogram downloaded into the
// caller's buffer by the slot's stream, so the host never copies samples.
#include <chrono>
#include <cmath>
#include <cstring>
#include <list>
#include <new>
#include <thread>
#include <unordered_map>
#include <vector>

#include "cwth_internal.h"

namespace {

constexpr uint32_t kServerMagic = 0x53565243u;  // "CRVS"

struct Key {
    double fs;
    int32_t S, hop;
    int64_t bucket;
    int32_t slot;  // -1: a plan every slot may share
    bool operator==(const Key& o) const {
        return fs == o.fs && S == o.S && hop == o.hop && bucket == o.bucket && slot == o.slot;
    }
};

struct KeyHash {
    size_t operator()(const Key& k) const {
        uint64_t f;
        memcpy(&f, &k.fs, sizeof(f));
        uint64_t h = f * 0x9E3779B97F4A7C15ull;
        h ^= (uint64_t)(uint32_t)k.S * 0xC2B2AE3D27D4EB4Full + (h << 6) + (h >> 2);
        h ^= (uint64_t)(uint32_t)k.hop * 0x165667B19E3779F9ull + (h << 6) + (h >> 2);
        h ^= (uint64_t)k.bucket * 0x27D4EB2F165667C5ull + (h << 6) + (h >> 2);
        h ^= (uint64_t)(uint32_t)(k.slot + 1) + (h << 6) + (h >> 2);
        return (size_t)h;
    }
};

struct CachedPlan {
    cwth_plan_t plan = nullptr;
    double bytes = 0;
    int64_t last_use = 0;
    int32_t busy = 0;
};

struct Pending {
    cwth_request r;
    int64_t bucket;
    // device address of r.x when it is page-locked (mapped into the
    // device's address space), else null
    const float* dx;
};

// One request of a batch as its gather kernel sees it.
struct IoEntry {
    const float* x;  // device address of the request's samples (host memory)
    int64_t n;
};

// Copies request i's samples from page-locked host memory into row i of
// the batch (and its length), reading them over the host link in place
// with 16-byte aligned float4 loads (a scalar head up to the source's
// alignment, a scalar tail).
__global__ void serve_gather(const IoEntry* __restrict__ tab, float* __restrict__ d_x, int64_t L,
                             int64_t* __restrict__ d_len) {
    const int i = blockIdx.y;
    const IoEntry e = tab[i];
    if (blockIdx.x == 0 && threadIdx.x == 0) d_len[i] = e.n;
    float* row = d_x + (int64_t)i * L;
    const int64_t head = (int64_t)((16 - ((uintptr_t)e.x & 15)) & 15) / 4;
    const int64_t h = head < e.n ? head : e.n;
    const int64_t t0 = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    const int64_t step = (int64_t)gridDim.x * blockDim.x;
    if (t0 < h) row[t0] = e.x[t0];
    const int64_t n4 = (e.n - h) / 4;
    const float4* x4 = reinterpret_cast<const float4*>(e.x + h);
    for (int64_t q = t0; q < n4; q += step) {
        const float4 v = x4[q];
        float* r = row + h + 4 * q;
        r[0] = v.x;
        r[1] = v.y;
        r[2] = v.z;
        r[3] = v.w;
    }
    for (int64_t t = h + 4 * n4 + t0; t < e.n; t += step) row[t] = e.x[t];
}

struct Slot {
    cudaStream_t st = nullptr;
    cudaEvent_t ev = nullptr;
    float* d_x = nullptr;
    size_t x_cap = 0;
    int64_t* d_len = nullptr;
    size_t len_cap = 0;
    float* d_out = nullptr;
    size_t out_cap = 0;
    uint8_t* d_stage = nullptr;  // bf16 staging of a direct-path batch (bound to the plan)
    size_t stage_cap = 0;
    int64_t* h_len = nullptr;  // page-locked
    size_t hlen_cap = 0;
    IoEntry* h_tab = nullptr;  // page-locked, read by the gather kernel
    IoEntry* d_tab = nullptr;  // its device address
    size_t tab_cap = 0;
    bool busy = false;
    int32_t status = CWTH_OK;
    std::vector<cwth_request> reqs;
    std::vector<Pending> io;
    Key plan_key{};
    double bytes = 0;
};

int64_t length_bucket(int64_t n) {
    int64_t b = int64_t(1) << 14;
    while (b < n) b <<= 1;
    return b;
}

double elapsed_s(std::chrono::steady_clock::time_point t0) {
    return std::chrono::duration<double>(std::chrono::steady_clock::now() - t0).count();
}

// Staging bytes of a batch: padded input rows, lengths, padded output.
double batch_bytes(int32_t b, int64_t L, int32_t S, int32_t hop) {
    const int64_t F = (L + hop - 1) / hop;
    return 4.0 * b * (double)L + 8.0 * b + 4.0 * b * (double)S * (double)F;
}

// Grows a slot buffer in stream order on the slot's own stream, whose
// previous batch has completed: unlike cudaFree, which waits for the whole
// device, this never stalls the other slots' batches.  The blocks come
// from the server's own memory pool, which keeps freed blocks mapped for
// reuse (no release at synchronisation points).  Capacity grows by at least
// half, so a slot meets few growths as its batches get larger.
template <class T>
cudaError_t grow_dev(T** p, size_t* cap, size_t need, cudaMemPool_t pool, cudaStream_t st) {
    if (*cap >= need) return cudaSuccess;
    const size_t n = std::max(need, *cap + *cap / 2);
    if (*p) cudaFreeAsync(*p, st);
    *p = nullptr;
    *cap = 0;
    cudaError_t e = cudaMallocFromPoolAsync((void**)p, n * sizeof(T), pool, st);
    if (e == cudaSuccess) *cap = n;
    return e;
}

}  // namespace

struct cwth_server_s {
    uint32_t magic = kServerMagic;
    int device = 0;
    cudaMemPool_t pool = nullptr;  // slot buffers
    cwth_server_config cfg{};
    std::chrono::steady_clock::time_point t0;
    std::list<Pending> pending;
    std::unordered_map<Key, CachedPlan, KeyHash> plans;
    std::vector<Slot> slots;
    std::vector<cwth_completion> ready;  // completions not yet handed out
    size_t ready_head = 0;
    double in_flight_bytes = 0, plan_bytes = 0, peak = 0;
    int64_t use_clock = 0, launched = 0, completed = 0, rejected = 0;
    int32_t evictions = 0;

    double used() const { return in_flight_bytes + plan_bytes; }
    void note_peak() { peak = std::max(peak, used()); }

    void complete(const cwth_request& r, int32_t status, int32_t b, double t) {
        cwth_completion c;
        c.rid = r.rid;
        c.status = status;
        c.batch_size = b;
        c.t_done = t;
        ready.push_back(c);
        ++completed;
    }

    // Scales of a key: S geometric centre frequencies from min(f_hi, fs/2)
    // down to f_lo, a_s = C fs / f_s.
    std::vector<double> scales(double fs, int32_t S) const {
        const double hi = std::min(cfg.f_hi, fs / 2.0);
        std::vector<double> a(S);
        for (int32_t s = 0; s < S; ++s) {
            const double f = S == 1 ? hi : hi * pow(cfg.f_lo / hi, (double)s / (double)(S - 1));
            a[s] = cfg.wavelet.center_freq * fs / f;
        }
        return a;
    }

    // Bytes of a batch's bf16 staging for the direct path (in its slot's
    // buffer); an estimate in dry-run mode, where no plan exists.
    double stage_bytes(const CachedPlan* cp, const Key& k, int32_t b) const {
        if (cfg.precision == CWTH_PREC_FP32 || cfg.path == CWTH_PATH_SPECTRAL) return 0.0;
        if (cfg.dry_run || !cp->plan) {
            const double parts = cfg.precision == CWTH_PREC_BF16 ? 1.0
                                 : (cfg.precision == CWTH_PREC_BF16X2 ? 2.0 : 3.0);
            return 2.0 * parts * b * (double)(k.bucket + 8192);
        }
        size_t n = 0;
        if (cwth_plan_stage_bytes(cp->plan, b, &n) != CWTH_OK) return 0.0;
        return (double)n;
    }

    // Evicts least recently used idle plans until `need` more bytes fit the
    // cache bound (or no idle plan is left).
    void make_room(double need) {
        while (plan_bytes + need > cfg.plan_cache_bytes) {
            auto victim = plans.end();
            for (auto it = plans.begin(); it != plans.end(); ++it)
                if (it->second.busy == 0 &&
                    (victim == plans.end() || it->second.last_use < victim->second.last_use))
                    victim = it;
            if (victim == plans.end()) return;
            if (victim->second.plan) cwth_destroy(victim->second.plan);
            plan_bytes -= victim->second.bytes;
            plans.erase(victim);
            ++evictions;
        }
    }

    // The cached plan for a key, made if needed, shared by all slots: a
    // batch with direct-path scales stages its bf16 signal in its slot's
    // own buffer, bound to the plan for that execute.
    cwth_status get_plan(const Pending& q, Key* key_out, CachedPlan** out) {
        Key k{q.r.fs, q.r.n_scales, q.r.hop, q.bucket, -1};
        *key_out = k;
        auto it = plans.find(k);
        if (it != plans.end()) {
            it->second.last_use = ++use_clock;
            *out = &it->second;
            return CWTH_OK;
        }
        CachedPlan cp;
        if (cfg.dry_run) {
            cp.bytes = cwth_server_plan_bytes(this, k.fs, k.S, k.hop, k.bucket);
        } else {
            const std::vector<double> a = scales(k.fs, k.S);
            cwth_status st = cwth_plan(&cfg.wavelet, a.data(), k.S, k.hop, k.fs, k.bucket,
                                       cfg.precision, cfg.path, &cp.plan);
            if (st != CWTH_OK) return st;
            cwth_plan_info info;
            st = cwth_plan_query(cp.plan, &info);
            if (st != CWTH_OK) {
                cwth_destroy(cp.plan);
                return st;
            }
            cp.bytes = (double)info.table_bytes + (double)info.workspace_bytes;
        }
        make_room(cp.bytes);
        cp.last_use = ++use_clock;
        plan_bytes += cp.bytes;
        note_peak();
        auto ins = plans.emplace(k, cp);
        *out = &ins.first->second;
        return CWTH_OK;
    }

    void retire(double t) {
        for (Slot& sl : slots) {
            if (!sl.busy) continue;
            if (!cfg.dry_run) {
                cudaError_t e = cudaEventQuery(sl.ev);
                if (e == cudaErrorNotReady) continue;
                if (e != cudaSuccess && sl.status == CWTH_OK) sl.status = CWTH_ERR_CUDA;
            }
            const int32_t b = (int32_t)sl.reqs.size();
            for (const cwth_request& r : sl.reqs) complete(r, sl.status, b, t);
            sl.reqs.clear();
            in_flight_bytes -= sl.bytes;
            auto it = plans.find(sl.plan_key);
            if (it != plans.end()) it->second.busy--;
            sl.busy = false;
        }
    }

    cwth_status launch(Slot& sl, CachedPlan* cp, const Key& key, std::vector<Pending>& sel,
                       double bytes) {
        cwth::NvtxRange nvtx_range("cwth_server_launch_batch");
        const int32_t b = (int32_t)sel.size();
        const int64_t L = key.bucket;
        const int64_t F = (L + key.hop - 1) / key.hop;
        sl.io.swap(sel);
        sl.reqs.clear();
        for (const Pending& q : sl.io) sl.reqs.push_back(q.r);
        sl.plan_key = key;
        sl.bytes = bytes;
        sl.status = CWTH_OK;
        sl.busy = true;
        cp->busy++;
        in_flight_bytes += bytes;
        note_peak();
        ++launched;
        if (cfg.dry_run) return CWTH_OK;
        cudaError_t e = grow_dev(&sl.d_x, &sl.x_cap, (size_t)b * (size_t)L, pool, sl.st);
        if (e == cudaSuccess) e = grow_dev(&sl.d_len, &sl.len_cap, (size_t)b, pool, sl.st);
        if (e == cudaSuccess)
            e = grow_dev(&sl.d_out, &sl.out_cap, (size_t)b * key.S * (size_t)F, pool, sl.st);
        // A batch with direct-path scales stages its bf16 signal in the
        // slot's buffer, bound to the (shared) plan for this execute.
        size_t need_stage = 0;
        if (e == cudaSuccess && cwth_plan_stage_bytes(cp->plan, b, &need_stage) == CWTH_OK &&
            need_stage > 0) {
            e = grow_dev(&sl.d_stage, &sl.stage_cap, need_stage, pool, sl.st);
            if (e == cudaSuccess &&
                cwth_plan_bind_stage(cp->plan, sl.d_stage, sl.stage_cap) != CWTH_OK)
                e = cudaErrorInvalidValue;
        }
        if (e == cudaSuccess && sl.hlen_cap < (size_t)b) {
            cudaFreeHost(sl.h_len);
            sl.h_len = nullptr;
            sl.hlen_cap = 0;
            e = cudaMallocHost(&sl.h_len, sizeof(int64_t) * (size_t)cfg.max_batch);
            if (e == cudaSuccess) sl.hlen_cap = (size_t)cfg.max_batch;
        }
        if (e == cudaSuccess && sl.tab_cap < (size_t)b) {
            cudaFreeHost(sl.h_tab);
            sl.h_tab = nullptr;
            sl.d_tab = nullptr;
            sl.tab_cap = 0;
            e = cudaMallocHost(&sl.h_tab, sizeof(IoEntry) * (size_t)cfg.max_batch);
            if (e == cudaSuccess) e = cudaHostGetDevicePointer((void**)&sl.d_tab, sl.h_tab, 0);
            if (e == cudaSuccess) sl.tab_cap = (size_t)cfg.max_batch;
        }
        // Page-locked inputs: one gather kernel reads the whole batch's
        // samples in place (no per-request upload call); others take one
        // upload each.  Scalograms go back by one copy-engine transfer per
        // request (measured faster than device stores into host memory).
        bool mapped = true;
        for (const Pending& q : sl.io) mapped = mapped && q.dx;
        if (mapped && e == cudaSuccess) {
            int64_t nmax = 0;
            for (int32_t i = 0; i < b; ++i) {
                const Pending& q = sl.io[i];
                sl.h_tab[i] = IoEntry{q.dx, q.r.n};
                nmax = std::max(nmax, q.r.n);
            }
            const int gx = (int)std::min<int64_t>(64, (nmax + 4095) / 4096);
            serve_gather<<<dim3(gx, b), 256, 0, sl.st>>>(sl.d_tab, sl.d_x, L, sl.d_len);
            e = cudaGetLastError();
            cwth_status st = e == cudaSuccess ? CWTH_OK : CWTH_ERR_CUDA;
            if (st == CWTH_OK)
                st = cwth_execute(cp->plan, sl.d_x, L, sl.d_len, b, sl.d_out, sl.st);
            for (int32_t i = 0; i < b && st == CWTH_OK; ++i) {
                const cwth_request& r = sl.reqs[i];
                const int64_t Fi = (r.n + key.hop - 1) / key.hop;
                if (cudaMemcpy2DAsync(r.out, sizeof(float) * (size_t)Fi,
                                      sl.d_out + (size_t)i * key.S * (size_t)F,
                                      sizeof(float) * (size_t)F, sizeof(float) * (size_t)Fi,
                                      (size_t)key.S, cudaMemcpyDeviceToHost, sl.st) != cudaSuccess)
                    st = CWTH_ERR_CUDA;
            }
            e = cudaEventRecord(sl.ev, sl.st);
            if (st == CWTH_OK && e != cudaSuccess) st = CWTH_ERR_CUDA;
            sl.status = st;
            return st;
        }
        for (int32_t i = 0; i < b && e == cudaSuccess; ++i) {
            const cwth_request& r = sl.reqs[i];
            sl.h_len[i] = r.n;
            e = cudaMemcpyAsync(sl.d_x + (size_t)i * L, r.x, sizeof(float) * (size_t)r.n,
                                cudaMemcpyHostToDevice, sl.st);
        }
        if (e == cudaSuccess)
            e = cudaMemcpyAsync(sl.d_len, sl.h_len, sizeof(int64_t) * (size_t)b,
                                cudaMemcpyHostToDevice, sl.st);
        cwth_status st = e == cudaSuccess ? CWTH_OK : CWTH_ERR_CUDA;
        if (st == CWTH_OK) st = cwth_execute(cp->plan, sl.d_x, L, sl.d_len, b, sl.d_out, sl.st);
        for (int32_t i = 0; i < b && st == CWTH_OK; ++i) {
            const cwth_request& r = sl.reqs[i];
            const int64_t Fi = (r.n + key.hop - 1) / key.hop;
            e = cudaMemcpy2DAsync(r.out, sizeof(float) * (size_t)Fi,
                                  sl.d_out + (size_t)i * key.S * (size_t)F, sizeof(float) * (size_t)F,
                                  sizeof(float) * (size_t)Fi, (size_t)key.S, cudaMemcpyDeviceToHost,
                                  sl.st);
            if (e != cudaSuccess) st = CWTH_ERR_CUDA;
        }
        // The event marks the batch done even after a failure part-way, so
        // the slot is retired once what was enqueued has run.
        e = cudaEventRecord(sl.ev, sl.st);
        if (st == CWTH_OK && e != cudaSuccess) st = CWTH_ERR_CUDA;
        sl.status = st;
        return st;
    }

    void admit(double t) {
        while (!pending.empty()) {
            int32_t slot = -1;
            for (size_t i = 0; i < slots.size(); ++i)
                if (!slots[i].busy) {
                    slot = (int32_t)i;
                    break;
                }
            if (slot < 0) return;
            // The oldest request and later ones of its key and bucket.
            const Pending& first = pending.front();
            std::vector<std::list<Pending>::iterator> pick;
            for (auto it = pending.begin(); it != pending.end() && (int32_t)pick.size() < cfg.max_batch;
                 ++it)
                if (it->bucket == first.bucket && it->r.hop == first.r.hop &&
                    it->r.n_scales == first.r.n_scales && it->r.fs == first.r.fs)
                    pick.push_back(it);
            Key key;
            CachedPlan* cp = nullptr;
            const cwth_status ps = get_plan(first, &key, &cp);
            if (ps != CWTH_OK) {
                for (auto it : pick) {
                    complete(it->r, ps, (int32_t)pick.size(), t);
                    pending.erase(it);
                }
                continue;
            }
            int32_t b = (int32_t)pick.size();
            double bytes = batch_bytes(b, key.bucket, key.S, key.hop) + stage_bytes(cp, key, b);
            while (b > 1 && used() + bytes > cfg.budget_bytes) {
                --b;
                bytes = batch_bytes(b, key.bucket, key.S, key.hop) + stage_bytes(cp, key, b);
            }
            if (used() + bytes > cfg.budget_bytes) {
                bool busy = false;
                for (const Slot& sl : slots) busy = busy || sl.busy;
                if (busy) return;  // wait for memory
                // Nothing in flight: evict idle plans other than this one,
                // then give up on the request if it still cannot fit.
                cp->busy++;
                make_room(cfg.plan_cache_bytes + 1.0);
                cp->busy--;
                if (used() + bytes > cfg.budget_bytes) {
                    complete(first.r, CWTH_ERR_OOM, 1, t);
                    ++rejected;
                    pending.erase(pick[0]);
                }
                continue;
            }
            std::vector<Pending> sel;
            sel.reserve(b);
            for (int32_t i = 0; i < b; ++i) {
                sel.push_back(*pick[i]);
                pending.erase(pick[i]);
            }
            launch(slots[slot], cp, key, sel, bytes);
        }
    }
};

extern "C" {

cwth_status cwth_server_create(const cwth_server_config* cfg, cwth_server_t* out) {
    if (out) *out = nullptr;
    if (!cfg || !out) return CWTH_ERR_INVALID_ARG;
    if (!(cfg->budget_bytes > 0) || !(cfg->plan_cache_bytes >= 0) || cfg->max_batch < 1 ||
        cfg->max_batch > 4096 || cfg->slots < 1 || cfg->slots > 64 ||
        cfg->precision < CWTH_PREC_FP32 || cfg->precision > CWTH_PREC_BF16X3 ||
        cfg->path < CWTH_PATH_AUTO || cfg->path > CWTH_PATH_DIRECT || !(cfg->f_lo > 0) ||
        !(cfg->f_hi >= cfg->f_lo) || !(cfg->wavelet.bandwidth > 0) ||
        !(cfg->wavelet.center_freq > 0))
        return CWTH_ERR_INVALID_ARG;
    cwth_server_s* s = new (std::nothrow) cwth_server_s();
    if (!s) return CWTH_ERR_OOM;
    s->cfg = *cfg;
    s->t0 = std::chrono::steady_clock::now();
    s->slots.resize(cfg->slots);
    if (!cfg->dry_run) {
        if (cudaGetDevice(&s->device) != cudaSuccess) {
            delete s;
            return CWTH_ERR_CUDA;
        }
        cudaMemPoolProps props;
        memset(&props, 0, sizeof(props));
        props.allocType = cudaMemAllocationTypePinned;
        props.handleTypes = cudaMemHandleTypeNone;
        props.location.type = cudaMemLocationTypeDevice;
        props.location.id = s->device;
        uint64_t keep = ~uint64_t(0);
        if (cudaMemPoolCreate(&s->pool, &props) != cudaSuccess ||
            cudaMemPoolSetAttribute(s->pool, cudaMemPoolAttrReleaseThreshold, &keep) != cudaSuccess) {
            cwth_server_destroy(s);
            return CWTH_ERR_CUDA;
        }
        for (Slot& sl : s->slots) {
            if (cudaStreamCreateWithFlags(&sl.st, cudaStreamNonBlocking) != cudaSuccess ||
                cudaEventCreateWithFlags(&sl.ev, cudaEventDisableTiming) != cudaSuccess) {
                cwth_server_destroy(s);
                return CWTH_ERR_CUDA;
            }
        }
    }
    *out = s;
    return CWTH_OK;
}

cwth_status cwth_server_submit(cwth_server_t s, const cwth_request* reqs, int32_t n) {
    if (!s || s->magic != kServerMagic || n < 0 || (n > 0 && !reqs)) return CWTH_ERR_INVALID_ARG;
    for (int32_t i = 0; i < n; ++i) {
        const cwth_request& r = reqs[i];
        if (!r.x || !r.out || r.n < 1 || !(r.fs > 0) || r.n_scales < 1 || r.hop < 1)
            return CWTH_ERR_INVALID_ARG;
    }
    for (int32_t i = 0; i < n; ++i) {
        Pending q{reqs[i], length_bucket(reqs[i].n), nullptr};
        if (!s->cfg.dry_run) {
            // Page-locked samples are read in place by the batch's gather
            // kernel (through their device address).
            cudaPointerAttributes ax;
            if (cudaPointerGetAttributes(&ax, reqs[i].x) == cudaSuccess &&
                ax.type == cudaMemoryTypeHost && ax.devicePointer)
                q.dx = static_cast<const float*>(ax.devicePointer);
            cudaGetLastError();  // a pageable pointer may leave an error behind
        }
        s->pending.push_back(q);
    }
    return CWTH_OK;
}

int32_t cwth_server_poll(cwth_server_t s, cwth_completion* done, int32_t max_done) {
    if (!s || s->magic != kServerMagic || max_done < 0 || (max_done > 0 && !done))
        return (int32_t)CWTH_ERR_INVALID_ARG * -1;
    const double t = elapsed_s(s->t0);
    s->retire(t);
    s->admit(t);
    int32_t k = 0;
    while (k < max_done && s->ready_head < s->ready.size()) done[k++] = s->ready[s->ready_head++];
    if (s->ready_head == s->ready.size()) {
        s->ready.clear();
        s->ready_head = 0;
    }
    return k;
}

cwth_status cwth_server_prepare(cwth_server_t s, double fs, int32_t n_scales, int32_t hop,
                                int64_t n_max) {
    if (!s || s->magic != kServerMagic || !(fs > 0) || n_scales < 1 || hop < 1 || n_max < 1)
        return CWTH_ERR_INVALID_ARG;
    cwth_request r;
    memset(&r, 0, sizeof(r));
    r.fs = fs;
    r.n_scales = n_scales;
    r.hop = hop;
    r.n = n_max;
    const Pending q{r, length_bucket(n_max), nullptr};
    Key key;
    CachedPlan* cp = nullptr;
    return s->get_plan(q, &key, &cp);
}

cwth_status cwth_server_stats_query(cwth_server_t s, cwth_server_stats* st) {
    if (!s || s->magic != kServerMagic || !st) return CWTH_ERR_INVALID_ARG;
    memset(st, 0, sizeof(*st));
    st->bytes_in_use = s->used();
    st->peak_bytes = s->peak;
    st->plan_bytes = s->plan_bytes;
    st->plans = (int32_t)s->plans.size();
    st->evictions = s->evictions;
    st->launched_batches = s->launched;
    st->completed = s->completed;
    st->rejected = s->rejected;
    st->pending = (int32_t)s->pending.size();
    int32_t f = 0;
    for (const Slot& sl : s->slots) f += sl.busy ? 1 : 0;
    st->in_flight = f;
    return CWTH_OK;
}

double cwth_server_plan_bytes(cwth_server_t s, double fs, int32_t n_scales, int32_t hop,
                              int64_t bucket) {
    if (!s || s->magic != kServerMagic || n_scales < 1 || hop < 1 || bucket < 1 || !(fs > 0))
        return -1.0;
    if (s->cfg.dry_run) {
        // Estimate: per-scale records and band tables, the twiddle table of
        // a 16384-sample segment, and for bf16 precisions a tap bank of up
        // to 4096 taps per scale part (batches stage in their slot's buffer).
        double b = 64.0 * n_scales + 8.0 * (16384 / 128 + 128) + 4096.0;
        if (s->cfg.precision != CWTH_PREC_FP32) b += 2.0 * 4096.0 * 2.0 * n_scales * 3.0;
        return b;
    }
    const std::vector<double> a = s->scales(fs, n_scales);
    cwth_plan_t p = nullptr;
    if (cwth_plan(&s->cfg.wavelet, a.data(), n_scales, hop, fs, bucket, s->cfg.precision,
                  s->cfg.path, &p) != CWTH_OK)
        return -1.0;
    cwth_plan_info info;
    double b = -1.0;
    if (cwth_plan_query(p, &info) == CWTH_OK)
        b = (double)info.table_bytes + (double)info.workspace_bytes;
    cwth_destroy(p);
    return b;
}

cwth_status cwth_server_replay(cwth_server_t s, const cwth_request* reqs, const double* arrival_s,
                               int32_t n, double* latency_s, int32_t* batch_sizes,
                               int32_t* status, double* wall_s) {
    if (!s || s->magic != kServerMagic || n < 0 || (n > 0 && (!reqs || !arrival_s)))
        return CWTH_ERR_INVALID_ARG;
    for (int32_t i = 1; i < n; ++i)
        if (arrival_s[i] < arrival_s[i - 1]) return CWTH_ERR_INVALID_ARG;
    std::unordered_map<int64_t, int32_t> index;
    index.reserve((size_t)n * 2);
    for (int32_t i = 0; i < n; ++i) index[reqs[i].rid] = i;
    if ((int32_t)index.size() != n) return CWTH_ERR_INVALID_ARG;  // ids must be unique
    const double start = elapsed_s(s->t0);
    std::vector<cwth_completion> buf(1024);
    int32_t next = 0, done = 0;
    while (done < n) {
        const double now = elapsed_s(s->t0) - start;
        int32_t k0 = next;
        while (next < n && arrival_s[next] <= now) ++next;
        if (next > k0) {
            cwth_status st = cwth_server_submit(s, reqs + k0, next - k0);
            if (st != CWTH_OK) return st;
        }
        const int32_t k = cwth_server_poll(s, buf.data(), (int32_t)buf.size());
        if (k < 0) return (cwth_status)(-k);
        for (int32_t j = 0; j < k; ++j) {
            auto it = index.find(buf[j].rid);
            if (it == index.end()) continue;
            const int32_t i = it->second;
            if (latency_s) latency_s[i] = buf[j].t_done - start - arrival_s[i];
            if (batch_sizes) batch_sizes[i] = buf[j].batch_size;
            if (status) status[i] = buf[j].status;
            ++done;
        }
        if (k == 0 && next < n && s->pending.empty()) {
            bool busy = false;
            for (const Slot& sl : s->slots) busy = busy || sl.busy;
            if (!busy) {
                // Idle until the next arrival (short sleeps keep the error small).
                const double wait = arrival_s[next] - (elapsed_s(s->t0) - start);
                if (wait > 2e-4) std::this_thread::sleep_for(std::chrono::microseconds(100));
            }
        }
    }
    if (wall_s) *wall_s = elapsed_s(s->t0) - start;
    return CWTH_OK;
}

cwth_status cwth_server_destroy(cwth_server_t s) {
    if (!s) return CWTH_OK;
    if (s->magic != kServerMagic) return CWTH_ERR_INVALID_ARG;
    for (Slot& sl : s->slots) {
        if (s->cfg.dry_run) break;
        if (sl.st) {
            // The slot buffers came from the stream-ordered allocator.
            if (sl.d_x) cudaFreeAsync(sl.d_x, sl.st);
            if (sl.d_len) cudaFreeAsync(sl.d_len, sl.st);
            if (sl.d_out) cudaFreeAsync(sl.d_out, sl.st);
            if (sl.d_stage) cudaFreeAsync(sl.d_stage, sl.st);
            cudaStreamSynchronize(sl.st);
        }
        if (sl.h_len) cudaFreeHost(sl.h_len);
        if (sl.h_tab) cudaFreeHost(sl.h_tab);
        if (sl.ev) cudaEventDestroy(sl.ev);
        if (sl.st) cudaStreamDestroy(sl.st);
    }
    if (s->pool) cudaMemPoolDestroy(s->pool);
    for (auto& kv : s->plans)
        if (kv.second.plan) cwth_destroy(kv.second.plan);
    s->magic = 0;
    delete s;
    return CWTH_OK;
}

}  // extern "C"
