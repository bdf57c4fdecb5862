// The batched step of the serving loop: every in-flight solve the kernels of
// the batched step can drive occupies a slot of a device work list, and one
// step of all of them is one launch per phase (the operator: FMA/CSR tiles
// and the tensor-core convolution units; the pivot-block solve; the update;
// the normalisation), each launch over flat (slot, tile) tables.  Slots of
// different sizes, steps j and targets k share every launch; a slot whose
// step counter reaches its k (or that broke down) drops out of the launches
// by itself.  The launch sequence of a turn (several steps) is captured in
// a CUDA graph once the composition of the batch has stayed the same for a
// turn, and replayed while it does.
//
// The operator of a PSF slot in BF16 is chosen by a project-written
// autotuner: the FMA column convolution, or the tensor-core convolution with
// one of several band heights (output rows per CTA), timed on the slot's own
// first basis vector the first time that (storage, PSF width, image size)
// is seen, and cached per process and in a JSON file (IPF_TUNE_CACHE).
#include <algorithm>
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <map>
#include <mutex>
#include <string>
#include <vector>

#include "ipf_internal.cuh"

namespace ipf {

namespace {

// ---------------------------------------------------------------------------
// autotuner
// ---------------------------------------------------------------------------
struct TuneChoice {
    int variant = 0;     // which kernel (e.g. 1: tensor-core convolution, 0: FMA)
    int param = 0;       // its tile parameter (e.g. output rows per unit)
    double us = 0.0;     // time of the chosen variant
};

struct Tuner {
    std::mutex mu;
    std::map<std::string, TuneChoice> table;
    bool loaded = false;
    std::string path;

    // (re)reads the file named by IPF_TUNE_CACHE when that name changes;
    // its entries replace the table's entries of the same keys
    void load() {
        const char* p = getenv("IPF_TUNE_CACHE");
        const std::string now = p ? p : "";
        if (loaded && now == path) return;
        loaded = true;
        path = now;
        if (path.empty()) return;
        FILE* f = fopen(p, "r");
        if (!f) return;
        std::string text;
        char buf[4096];
        size_t got;
        while ((got = fread(buf, 1, sizeof buf, f)) > 0) text.append(buf, got);
        fclose(f);
        // entries: {"key": "...", "variant": V, "param": P, "us": T}
        size_t at = 0;
        while ((at = text.find("\"key\": \"", at)) != std::string::npos) {
            at += 8;
            const size_t end = text.find('"', at);
            if (end == std::string::npos) break;
            const std::string key = text.substr(at, end - at);
            TuneChoice c;
            const size_t va = text.find("\"variant\": ", end);
            const size_t pa = text.find("\"param\": ", end);
            const size_t us = text.find("\"us\": ", end);
            if (va == std::string::npos || pa == std::string::npos || us == std::string::npos) break;
            c.variant = atoi(text.c_str() + va + 11);
            c.param = atoi(text.c_str() + pa + 9);
            c.us = atof(text.c_str() + us + 6);
            table[key] = c;
            at = end;
        }
    }

    void save() {
        if (path.empty()) return;
        const std::string tmp = path + ".tmp";
        FILE* f = fopen(tmp.c_str(), "w");
        if (!f) return;
        fprintf(f, "{\"version\": 1, \"entries\": [\n");
        size_t i = 0;
        for (const auto& kv : table) {
            fprintf(f, "  {\"key\": \"%s\", \"variant\": %d, \"param\": %d, \"us\": %.3f}%s\n",
                    kv.first.c_str(), kv.second.variant, kv.second.param, kv.second.us,
                    ++i < table.size() ? "," : "");
        }
        fprintf(f, "]}\n");
        fclose(f);
        rename(tmp.c_str(), path.c_str());
    }
};

Tuner& tuner() {
    static Tuner t;
    return t;
}

std::string tune_key(int storage, const OpDev& op) {
    char b[96];
    snprintf(b, sizeof b, "conv/%s/kw%d/%dx%d", storage == IPF_STORE_BF16 ? "bf16" : "other", op.kw, op.rows,
             op.cols);
    return b;
}

int cdiv(long long a, long long b) { return (int)((a + b - 1) / b); }

}  // namespace

bool tune_lookup(const char* key, int* variant, int* param) {
    Tuner& tn = tuner();
    std::lock_guard<std::mutex> lk(tn.mu);
    tn.load();
    auto it = tn.table.find(key);
    if (it == tn.table.end()) return false;
    *variant = it->second.variant;
    *param = it->second.param;
    return true;
}

void tune_store(const char* key, int variant, int param, double us) {
    Tuner& tn = tuner();
    std::lock_guard<std::mutex> lk(tn.mu);
    tn.load();
    TuneChoice c;
    c.variant = variant;
    c.param = param;
    c.us = us;
    tn.table[key] = c;
    tn.save();
}

// ---------------------------------------------------------------------------
// the engine
// ---------------------------------------------------------------------------
struct BatchEngine {
    struct Slot {
        bool used = false;
        ipf_ctx* ctx = nullptr;
        SlotDesc d{};
        int storage = 0;                 // the slot's storage type (F32, BF16, F16)
        int steps = 0;                   // steps enqueued for this slot
    };
    struct Stage {
        void* host = nullptr;
        size_t bytes = 0;
        cudaEvent_t ev = nullptr;
    };
    int num_sms = 1;
    cudaStream_t s = nullptr, s2 = nullptr;   // the step's stream, and the pivot branch beside the operator
    cudaEvent_t ev_ready = nullptr, ev_t0 = nullptr, ev_t1 = nullptr, ev_fork = nullptr, ev_join = nullptr;
    Slot slots[kMaxSlots];
    std::vector<unsigned char> maps;     // kMaxSlots tensor maps, host (passed by value at launch)
    SlotDesc* d_slots = nullptr;         // kMaxSlots entries
    SlotDesc* d_tune = nullptr;          // kMaxSlots entries, for the tuner's one-slot tables
    int* d_groups = nullptr;             // kMaxSlots x kCsrGroupRec: CSR slots sharing one matrix
    unsigned char* d_stage = nullptr;    // the groups' staging rows of v_j
    size_t stage_cap = 0;
    TileRef* d_tiles = nullptr;
    size_t tile_cap = 0;
    unsigned epoch = 1, uploaded_epoch = 0, ran_epoch = 0;
    int ran_turns = 0;                         // eager turns of the composition ran_epoch
    static constexpr int kEagerTurnsBeforeCapture = 3;
    Stage stage[4];
    int stage_next = 0;
    cudaGraphExec_t gexec = nullptr;
    unsigned gexec_epoch = 0;
    int gexec_steps = 0;
    long long graph_turns = 0, eager_turns = 0, captures = 0;

    int used() const {
        int c = 0;
        for (const Slot& sl : slots) c += sl.used ? 1 : 0;
        return c;
    }

    // copy bytes to the device through a pinned staging buffer (ring of 4,
    // each reused only after its previous copy has completed)
    cudaError_t stage_copy(void* dst, const void* src, size_t bytes) {
        Stage& st = stage[stage_next];
        stage_next = (stage_next + 1) % 4;
        cudaError_t e;
        if (st.ev && (e = cudaEventSynchronize(st.ev)) != cudaSuccess) return e;
        if (st.bytes < bytes) {
            if (st.host) cudaFreeHost(st.host);
            st.host = nullptr;
            st.bytes = 0;
            if ((e = cudaMallocHost(&st.host, bytes)) != cudaSuccess) return e;
            st.bytes = bytes;
        }
        if (!st.ev && (e = cudaEventCreateWithFlags(&st.ev, cudaEventDisableTiming)) != cudaSuccess) return e;
        memcpy(st.host, src, bytes);
        if ((e = cudaMemcpyAsync(dst, st.host, bytes, cudaMemcpyHostToDevice, s)) != cudaSuccess) return e;
        return cudaEventRecord(st.ev, s);
    }

    // the (slot, tile) tables of the current composition, to the device:
    // per storage group (FP32, BF16, FP16) the operator tiles, the
    // tensor-core units (BF16: KP 16 and 32), the slot list of the pivot
    // solve, the update, the normalisation tiles, the products at the pivot
    // rows and the CSR tiles of slot groups sharing one matrix (each row's
    // nonzeros read once for up to kCsrGroup slots)
    static constexpr int kGroups = 3;
    static constexpr int kTables = 9;        // op, tc16, tc32, piv, upd, norm, pivot-row products, CSR groups,
                                             // CSR staging
    struct Group {
        int storage = 0;
        int count[kTables] = {0};
        size_t off[kTables] = {0};
        int k_max = 0, m_s_max = 0;
    };
    Group grp[kGroups];

    cudaError_t upload() {
        std::vector<SlotDesc> hs(kMaxSlots);
        memset(hs.data(), 0, hs.size() * sizeof(SlotDesc));
        std::vector<TileRef> tab[kGroups][kTables];
        std::vector<int> hg((size_t)kMaxSlots * kCsrGroupRec, 0);
        size_t stage_bytes = 0;
        int ngroups = 0;
        std::vector<int> csr[kGroups];
        for (int g = 0; g < kGroups; ++g) grp[g] = Group();
        for (int i = 0; i < kMaxSlots; ++i) {
            const Slot& sl = slots[i];
            if (!sl.used) continue;
            const SlotDesc& d = sl.d;
            hs[i] = d;
            const int g = sl.storage - IPF_STORE_F32;
            Group& G = grp[g];
            G.storage = sl.storage;
            G.k_max = std::max(G.k_max, d.g.k_max);
            G.m_s_max = std::max(G.m_s_max, d.sp.m_s);
            std::vector<TileRef>* t = tab[g];
            if (d.tc_kp) {
                std::vector<TileRef>& u = t[d.tc_kp == 32 ? 2 : 1];
                for (int q = 0, nq = d.tc_ct * cdiv(d.op.rows, d.tc_rows); q < nq; ++q) u.push_back({i, q});
            } else if (d.op.kind == IPF_OP_CSR) {
                csr[g].push_back(i);
            } else {
                for (int q = 0, nq = d.conv_cols * cdiv(d.op.rows, 16); q < nq; ++q) t[0].push_back({i, q});
            }
            t[3].push_back({i, 0});
            for (int q = 0, nq = cdiv(d.g.N, kBatchUpdTile); q < nq; ++q) t[4].push_back({i, q});
            for (int q = 0; q < d.norm_tiles; ++q) t[5].push_back({i, q});
            // pivot-row tiles: 8 CSR rows (a warp each) or 2 PSF rows (four warps each)
            for (int q = 0, nq = cdiv(d.g.k_max + 1, d.op.kind == IPF_OP_CSR ? 8 : 2); q < nq; ++q)
                t[6].push_back({i, q});
        }
        // CSR slots of one storage type on the same matrix, in groups of up
        // to kCsrGroup (slot order), one tile list per group
        for (int g = 0; g < kGroups; ++g) {
            std::vector<int>& c = csr[g];
            std::vector<char> done(c.size(), 0);
            for (size_t a = 0; a < c.size(); ++a) {
                if (done[a]) continue;
                const OpDev& oa = slots[c[a]].d.op;
                int* gr = hg.data() + (size_t)ngroups * kCsrGroupRec;
                gr[0] = 0;
                for (size_t b = a; b < c.size() && gr[0] < kCsrGroup; ++b) {
                    const OpDev& ob = slots[c[b]].d.op;
                    if (done[b] || ob.rowptr != oa.rowptr || ob.colind != oa.colind || ob.vals != oa.vals ||
                        ob.rows != oa.rows)
                        continue;
                    done[b] = 1;
                    gr[1 + gr[0]++] = c[b];
                }
                for (int q = 0, nq = cdiv(oa.rows, kBatchCsrRows); q < nq; ++q) tab[g][7].push_back({ngroups, q});
                for (int q = 0, nq = cdiv(oa.cols, 1024); q < nq; ++q) tab[g][8].push_back({ngroups, q});
                // staging rows: cols x kCsrGroup values, 256-byte aligned
                const size_t es = grp[g].storage == IPF_STORE_F32 ? 4 : 2;
                gr[kCsrGroup + 1] = (int)(unsigned)(stage_bytes & 0xFFFFFFFFu);
                gr[kCsrGroup + 2] = (int)(unsigned)(stage_bytes >> 32);
                stage_bytes += ((size_t)oa.cols * kCsrGroup * es + 255) / 256 * 256;
                ++ngroups;
            }
        }
        std::vector<TileRef> all;
        for (int g = 0; g < kGroups; ++g)
            for (int q = 0; q < kTables; ++q) {
                grp[g].off[q] = all.size();
                grp[g].count[q] = (int)tab[g][q].size();
                all.insert(all.end(), tab[g][q].begin(), tab[g][q].end());
            }
        const size_t total = all.size();
        cudaError_t e;
        if (total > tile_cap) {
            // the old table may still be read by launches in flight
            if ((e = cudaStreamSynchronize(s)) != cudaSuccess) return e;
            if (d_tiles) cudaFree(d_tiles);
            d_tiles = nullptr;
            tile_cap = 0;
            const size_t cap = std::max(total * 2, (size_t)1 << 16);
            if ((e = cudaMalloc(&d_tiles, cap * sizeof(TileRef))) != cudaSuccess) return e;
            tile_cap = cap;
        }
        if ((e = stage_copy(d_slots, hs.data(), hs.size() * sizeof(SlotDesc))) != cudaSuccess) return e;
        if (stage_bytes > stage_cap) {
            // the old staging rows may still be read by launches in flight
            if ((e = cudaStreamSynchronize(s)) != cudaSuccess) return e;
            if (d_stage) cudaFree(d_stage);
            d_stage = nullptr;
            stage_cap = 0;
            if ((e = cudaMalloc(&d_stage, stage_bytes * 2)) != cudaSuccess) return e;
            stage_cap = stage_bytes * 2;
        }
        if (ngroups && (e = stage_copy(d_groups, hg.data(), (size_t)ngroups * kCsrGroupRec * sizeof(int))) !=
                           cudaSuccess)
            return e;
        if (total && (e = stage_copy(d_tiles, all.data(), total * sizeof(TileRef))) != cudaSuccess) return e;
        uploaded_epoch = epoch;
        return cudaSuccess;
    }

    // one batched step of every slot of the uploaded composition: the
    // products at the pivot rows and the FP64 pivot-block solve on the
    // second stream beside the operator (they need only v_j and the
    // pivots), joined before the update that consumes both
    cudaError_t step_launches() {
        cudaError_t e;
        if ((e = cudaEventRecord(ev_fork, s)) != cudaSuccess) return e;
        if ((e = cudaStreamWaitEvent(s2, ev_fork, 0)) != cudaSuccess) return e;
        for (const Group& G : grp) {
            if (!G.count[3]) continue;
            TileRef* t = d_tiles;
            if ((e = launch_batch_pivot_rows(G.storage, d_slots, t + G.off[6], G.count[6], num_sms, s2)) != cudaSuccess)
                return e;
            if ((e = launch_batch_pivot_solve(G.storage, d_slots, t + G.off[3], G.count[3], G.k_max, s2)) !=
                cudaSuccess)
                return e;
        }
        if ((e = cudaEventRecord(ev_join, s2)) != cudaSuccess) return e;
        for (const Group& G : grp) {
            if (!G.count[3]) continue;
            const int st = G.storage;
            TileRef* t = d_tiles;
            if ((e = launch_batch_operator(st, d_slots, t + G.off[0], G.count[0], num_sms, s)) != cudaSuccess) return e;
            if ((e = launch_batch_csr_group(st, d_slots, d_groups, d_stage, t + G.off[8], G.count[8], t + G.off[7],
                                            G.count[7], num_sms, s)) != cudaSuccess)
                return e;
            if ((e = launch_batch_conv_tc(16, maps.data(), d_slots, t + G.off[1], G.count[1], s)) != cudaSuccess)
                return e;
            if ((e = launch_batch_conv_tc(32, maps.data(), d_slots, t + G.off[2], G.count[2], s)) != cudaSuccess)
                return e;
        }
        if ((e = cudaStreamWaitEvent(s, ev_join, 0)) != cudaSuccess) return e;
        for (const Group& G : grp) {
            if (!G.count[3]) continue;
            const int st = G.storage;
            TileRef* t = d_tiles;
            if ((e = launch_batch_update(st, d_slots, t + G.off[4], G.count[4], G.k_max, G.m_s_max, num_sms, s)) !=
                cudaSuccess)
                return e;
            if ((e = launch_batch_normalize(st, d_slots, t + G.off[5], G.count[5], num_sms, s)) != cudaSuccess)
                return e;
        }
        return cudaSuccess;
    }

    // ms per product of one operator variant on slot i (its first basis
    // vector; only w is written, which the slot's first step overwrites)
    TileRef* d_tune_tiles = nullptr;
    size_t tune_cap = 0;
    cudaError_t time_variant(int i, const SlotDesc& d, double* ms) {
        std::vector<TileRef> t;
        if (d.tc_kp)
            for (int u = 0, nu = d.tc_ct * cdiv(d.op.rows, d.tc_rows); u < nu; ++u) t.push_back({i, u});
        else
            for (int u = 0, nu = d.conv_cols * cdiv(d.op.rows, 16); u < nu; ++u) t.push_back({i, u});
        cudaError_t e;
        if (t.size() > tune_cap) {
            if ((e = cudaStreamSynchronize(s)) != cudaSuccess) return e;
            if (d_tune_tiles) cudaFree(d_tune_tiles);
            d_tune_tiles = nullptr;
            tune_cap = 0;
            if ((e = cudaMalloc(&d_tune_tiles, t.size() * 2 * sizeof(TileRef))) != cudaSuccess) return e;
            tune_cap = t.size() * 2;
        }
        if ((e = stage_copy(d_tune + i, &d, sizeof(SlotDesc))) != cudaSuccess) return e;
        if ((e = stage_copy(d_tune_tiles, t.data(), t.size() * sizeof(TileRef))) != cudaSuccess) return e;
        auto go = [&]() {
            return d.tc_kp ? launch_batch_conv_tc(d.tc_kp, maps.data(), d_tune, d_tune_tiles, (int)t.size(), s)
                           : launch_batch_operator(IPF_STORE_BF16, d_tune, d_tune_tiles, (int)t.size(), num_sms, s);
        };
        constexpr int kReps = 3;
        if ((e = go()) != cudaSuccess) return e;
        if ((e = cudaEventRecord(ev_t0, s)) != cudaSuccess) return e;
        for (int r = 0; r < kReps; ++r)
            if ((e = go()) != cudaSuccess) return e;
        if ((e = cudaEventRecord(ev_t1, s)) != cudaSuccess) return e;
        if ((e = cudaEventSynchronize(ev_t1)) != cudaSuccess) return e;
        float t_ms = 0.f;
        if ((e = cudaEventElapsedTime(&t_ms, ev_t0, ev_t1)) != cudaSuccess) return e;
        *ms = t_ms / kReps;
        return cudaSuccess;
    }

    // the operator of a BF16 PSF slot whose PSF has a tensor-core operand:
    // the tuned choice for its (width, image size), measured here if new
    cudaError_t choose_operator(int i, SlotDesc* d) {
        const std::string key = tune_key(IPF_STORE_BF16, d->op);
        Tuner& tn = tuner();
        {
            std::lock_guard<std::mutex> lk(tn.mu);
            tn.load();
            auto it = tn.table.find(key);
            if (it != tn.table.end()) {
                if (it->second.variant == 1 && it->second.param > 0) {
                    d->tc_kp = d->op.tc_kp;
                    d->tc_rows = it->second.param;
                }
                return cudaSuccess;
            }
        }
        TuneChoice best;
        double ms = 0.0;
        SlotDesc c = *d;
        c.tc_kp = 0;
        cudaError_t e = time_variant(i, c, &ms);
        if (e != cudaSuccess) return e;
        best.us = ms * 1e3;
        for (int rows : {32, 64, 128, 256}) {
            if (rows > d->op.rows && rows != 32) break;
            c.tc_kp = d->op.tc_kp;
            c.tc_rows = rows;
            if ((e = time_variant(i, c, &ms)) != cudaSuccess) return e;
            if (ms * 1e3 < best.us) {
                best.us = ms * 1e3;
                best.variant = 1;
                best.param = rows;
            }
        }
        {
            std::lock_guard<std::mutex> lk(tn.mu);
            tn.table[key] = best;
            tn.save();
        }
        if (best.variant == 1) {
            d->tc_kp = d->op.tc_kp;
            d->tc_rows = best.param;
        }
        return cudaSuccess;
    }
};

BatchEngine* batch_create() {
    BatchEngine* b = new BatchEngine();
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e == cudaSuccess) e = cudaDeviceGetAttribute(&b->num_sms, cudaDevAttrMultiProcessorCount, dev);
    int lo = 0, hi = 0;
    if (e == cudaSuccess) e = cudaDeviceGetStreamPriorityRange(&lo, &hi);
    if (e == cudaSuccess) e = cudaStreamCreateWithPriority(&b->s, cudaStreamNonBlocking, lo);
    if (e == cudaSuccess) e = cudaStreamCreateWithPriority(&b->s2, cudaStreamNonBlocking, hi);
    if (e == cudaSuccess) e = cudaEventCreateWithFlags(&b->ev_ready, cudaEventDisableTiming);
    if (e == cudaSuccess) e = cudaEventCreateWithFlags(&b->ev_fork, cudaEventDisableTiming);
    if (e == cudaSuccess) e = cudaEventCreateWithFlags(&b->ev_join, cudaEventDisableTiming);
    if (e == cudaSuccess) e = cudaEventCreate(&b->ev_t0);
    if (e == cudaSuccess) e = cudaEventCreate(&b->ev_t1);
    if (e == cudaSuccess) e = cudaMalloc(&b->d_slots, sizeof(SlotDesc) * kMaxSlots);
    if (e == cudaSuccess) e = cudaMalloc(&b->d_tune, sizeof(SlotDesc) * kMaxSlots);
    if (e == cudaSuccess) e = cudaMalloc(&b->d_groups, sizeof(int) * kMaxSlots * kCsrGroupRec);
    if (e == cudaSuccess) e = cudaMemsetAsync(b->d_slots, 0, sizeof(SlotDesc) * kMaxSlots, b->s);
    if (e == cudaSuccess) e = cudaMemsetAsync(b->d_tune, 0, sizeof(SlotDesc) * kMaxSlots, b->s);
    if (e != cudaSuccess) {
        batch_destroy(b);
        return nullptr;
    }
    b->maps.assign(kMaxSlots * conv_tc_map_bytes(), 0);
    return b;
}

void batch_destroy(BatchEngine* b) {
    if (!b) return;
    if (b->s) cudaStreamSynchronize(b->s);
    if (b->gexec) cudaGraphExecDestroy(b->gexec);
    for (auto& st : b->stage) {
        if (st.ev) cudaEventDestroy(st.ev);
        if (st.host) cudaFreeHost(st.host);
    }
    if (b->d_tiles) cudaFree(b->d_tiles);
    if (b->d_tune_tiles) cudaFree(b->d_tune_tiles);
    if (b->d_slots) cudaFree(b->d_slots);
    if (b->d_tune) cudaFree(b->d_tune);
    if (b->d_groups) cudaFree(b->d_groups);
    if (b->d_stage) cudaFree(b->d_stage);
    if (b->ev_ready) cudaEventDestroy(b->ev_ready);
    if (b->ev_t0) cudaEventDestroy(b->ev_t0);
    if (b->ev_t1) cudaEventDestroy(b->ev_t1);
    if (b->ev_fork) cudaEventDestroy(b->ev_fork);
    if (b->ev_join) cudaEventDestroy(b->ev_join);
    if (b->s2) cudaStreamSynchronize(b->s2);
    if (b->s2) cudaStreamDestroy(b->s2);
    if (b->s) cudaStreamDestroy(b->s);
    delete b;
}

int batch_add(BatchEngine* b, ipf_ctx* c, int k, cudaStream_t ready) {
    SlotDesc d;
    int stg = 0;
    if (!b || k < 1 || !ctx_slot_desc(c, &d, &stg)) return -1;
    int i = 0;
    while (i < kMaxSlots && b->slots[i].used) ++i;
    if (i == kMaxSlots) return -1;
    // the slot's initialisation (on its context's streams, ordered before
    // `ready`) completes before any batched step reads it
    if (cudaEventRecord(b->ev_ready, ready) != cudaSuccess || cudaStreamWaitEvent(b->s, b->ev_ready, 0) != cudaSuccess)
        return -1;
    d.k_target = k < d.g.k_max ? k : d.g.k_max;
    d.norm_tiles = cdiv(d.g.n, kBatchNormTile);
    d.conv_cols = d.op.kind == IPF_OP_PSF2D ? cdiv(d.op.cols, 128) : 0;
    d.tc_ct = d.op.kind == IPF_OP_PSF2D ? cdiv(d.op.cols, 128) : 0;
    if (d.op.kind == IPF_OP_PSF2D && stg == IPF_STORE_BF16 && d.op.tc_kp &&
        conv_tc_map(d.op, d.bf.V, d.g.ldv, d.g.k_max + 1, b->maps.data() + (size_t)i * conv_tc_map_bytes())) {
        if (b->choose_operator(i, &d) != cudaSuccess) return -1;
    }
    BatchEngine::Slot& sl = b->slots[i];
    sl.used = true;
    sl.ctx = c;
    sl.d = d;
    sl.storage = stg;
    sl.steps = 0;
    ++b->epoch;
    return i;
}

void batch_remove(BatchEngine* b, int i) {
    if (!b || i < 0 || i >= kMaxSlots || !b->slots[i].used) return;
    b->slots[i] = BatchEngine::Slot();
    ++b->epoch;
}

int batch_steps(const BatchEngine* b, int i) { return (b && i >= 0 && i < kMaxSlots) ? b->slots[i].steps : 0; }

int batch_used(const BatchEngine* b) { return b ? b->used() : 0; }

// enqueue `steps` batched steps of every slot (a turn) on the engine
// stream, and record `done` after them; each slot's step count advances
cudaError_t batch_run(BatchEngine* b, int steps, cudaEvent_t done) {
    if (!b || steps < 1) return cudaErrorInvalidValue;
    cudaError_t e;
    if (b->used() > 0) {
        if (b->uploaded_epoch != b->epoch && (e = b->upload()) != cudaSuccess) return e;
        const bool reuse = b->gexec && b->gexec_epoch == b->epoch && b->gexec_steps == steps;
        if (reuse) {
            if ((e = cudaGraphLaunch(b->gexec, b->s)) != cudaSuccess) return e;
            ++b->graph_turns;
        } else if (b->ran_epoch == b->epoch && b->ran_turns >= BatchEngine::kEagerTurnsBeforeCapture) {
            // the composition held for several turns: capture it (under
            // churn, a capture and instantiation costs more host time than
            // the eager turns it would replace)
            cudaGraph_t g = nullptr;
            if ((e = cudaStreamBeginCapture(b->s, cudaStreamCaptureModeRelaxed)) != cudaSuccess) return e;
            cudaError_t e1 = cudaSuccess;
            for (int t = 0; t < steps && e1 == cudaSuccess; ++t) e1 = b->step_launches();
            cudaError_t e2 = cudaStreamEndCapture(b->s, &g);
            if (e1 != cudaSuccess) { if (g) cudaGraphDestroy(g); return e1; }
            if (e2 != cudaSuccess) return e2;
            if (b->gexec) cudaGraphExecDestroy(b->gexec);
            b->gexec = nullptr;
            e = cudaGraphInstantiate(&b->gexec, g, 0);
            cudaGraphDestroy(g);
            if (e != cudaSuccess) return e;
            b->gexec_epoch = b->epoch;
            b->gexec_steps = steps;
            ++b->captures;
            if ((e = cudaGraphLaunch(b->gexec, b->s)) != cudaSuccess) return e;
            ++b->graph_turns;
        } else {
            for (int t = 0; t < steps; ++t)
                if ((e = b->step_launches()) != cudaSuccess) return e;
            b->ran_turns = b->ran_epoch == b->epoch ? b->ran_turns + 1 : 1;
            b->ran_epoch = b->epoch;
            ++b->eager_turns;
        }
        for (auto& sl : b->slots)
            if (sl.used) sl.steps += steps;
    }
    return cudaEventRecord(done, b->s);
}

void batch_counters(const BatchEngine* b, long long* graph_turns, long long* eager_turns, long long* captures) {
    if (!b) return;
    if (graph_turns) *graph_turns = b->graph_turns;
    if (eager_turns) *eager_turns = b->eager_turns;
    if (captures) *captures = b->captures;
}

}  // namespace ipf
