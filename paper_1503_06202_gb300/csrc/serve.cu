// serve.cu -- the streaming service: continuous batching of frame blocks from
// many concurrent streams into device-resident integrations (paper Sec. IV-A
// data flow and Sec. IV-C-1 integration, on one GPU).
//
// Each admitted stream owns, in device memory, its int32 accumulators, two
// dump buffers and two slices of decode planes (room for `max_blocks` blocks).
// Admission charges all of these against the server's HBM budget (and, if
// asked, the stream's compute demand against a compute budget); a refused
// stream can be admitted later, once others close and free their share.
//
// A worker thread runs the loop.  Each round it takes, from every stream with
// queued blocks, up to `max_blocks` of them (never across a dump boundary) --
// blocks that arrived while earlier rounds were on the GPU join the next round.
// A stream whose blocks a single-pass kernel takes (N a multiple of 16 up to the
// build's bound, every block 16-byte aligned, blocks a whole number of the
// kernel's stages and at most 32,768 samples) gets single-pass launches that
// read its blocks where they are, one tensor map per block, and add into its
// accumulators (or store, for the first round of an integration): no planes.
// The other streams' blocks are decoded with one persistent TMA launch
// (per-block tensor maps; a thread-per-row launch only for blocks TMA cannot
// address) into their plane slices and correlated with one persistent
// tensor-core launch over all of their tiles.  The environment variable
// XENG_FUSED_KERNEL (read at creation) forces a single-pass kernel as for a
// handle; "none" sends every stream through the planes.  A stream whose integration reaches `dump_samples` gets a
// device copy of its accumulators queued into a free dump buffer right after
// the round, and starts a fresh integration.  Two rounds may be in flight; the
// worker polls their events, marks blocks consumed, publishes dumps and
// records latencies: block arrival -> block integrated, and last block of an
// integration -> its dump available.
//
// Lost and late blocks (Sec. IV-A: momentary faults must not stop the data
// gathering).  Block number b of a stream belongs to integration
// b / (dump_samples / block_samples).  Blocks may arrive with gaps; an
// integration closes when all its blocks are in, when a block of a later
// integration reaches the head of the stream's queue, or on xserve_flush --
// then it is dumped with the samples it has, and the dump reports how many
// blocks it holds and how many are missing.  A block of an integration that a
// later block has already closed is refused (XENG_ERR_LATE) and counted.
#include <algorithm>
#include <chrono>
#include <condition_variable>
#include <cstring>
#include <deque>
#include <mutex>
#include <new>
#include <thread>
#include <vector>

#include "../../include/xeng.h"
#include "xeng_internal.h"

using namespace xeng;

namespace {

double now_s()
{
    using namespace std::chrono;
    return duration<double>(steady_clock::now().time_since_epoch()).count();
}

struct QBlock {
    const uint8_t *ptr;  // nullptr: a flush marker (close the integration here)
    double arrival;
    int64_t integ;       // integration the block belongs to
};

struct DumpSlot {
    int32_t *buf = nullptr;
    bool busy = false;       // written or being written, not yet taken by the client
    bool ready = false;      // the copy has completed
    int64_t samples = 0;
    double last_arrival = 0, ready_time = 0;
    int64_t seq = 0;         // integration number of the stream
    int64_t blocks = 0;      // blocks integrated
};

struct SStream {
    bool open = false;
    int id = -1;
    int32_t N = 0, F = 0;
    int64_t dump_samples = 0, block_samples = 0, bs_pad = 0;
    int single = 0;                  // single-pass kernel of the stream's rounds (no planes), else 0
    int64_t n_pad = 0;
    double demand_tops = 0;
    int64_t bytes = 0;               // charged to the HBM budget
    int32_t *acc = nullptr;
    uint8_t *planes[2] = {nullptr, nullptr};
    int2 *partials[2] = {nullptr, nullptr};  // raw-nibble rounds: per-tile nibble sums of the slice
    int2 *sums[2] = {nullptr, nullptr};      // ... and their totals (S, D) per [F][n_pad]
    DumpSlot dump[2];
    bool fresh = true;
    int64_t integrated = 0;          // samples in the current integration (launched)
    double last_arrival = 0;         // of the current integration's latest launched block
    int64_t cur_integ = 0;           // integration the worker is filling
    std::deque<QBlock> queue;
    int64_t submitted = 0, consumed = 0;
    int64_t inflight = 0;            // blocks in rounds not yet complete
    // submission side: the newest integration a block was submitted for, and
    // which of its blocks have come (a block number may be submitted once)
    int64_t top_integ = 0, next_block = 0;
    std::vector<uint8_t> seen;
    int64_t blocks_per_dump() const { return dump_samples / block_samples; }
};

struct Round {
    cudaEvent_t ev = nullptr;
    cudaEvent_t t0 = nullptr, t1 = nullptr, t2 = nullptr;  // timing: round start, decode done, correlate done
    int slot = 0;
    struct Part { int stream; int nblocks; std::vector<double> arrivals; int dump_slot; };
    // streams of the round on the single-pass kernels: kernel, first map in the
    // slot's table, blocks, and whether the round stores (first of an integration)
    struct Single { int stream; int kernel; int64_t map0; int nblocks; bool store; };
    std::vector<Single> singles;
    std::vector<Part> parts;
    double useful_ops = 0;
};

}  // namespace

struct xserve_s {
    xserve_opts_t opts{};
    int device = 0, num_sms = 0;
    int64_t used_bytes = 0;
    double used_tops = 0;
    std::vector<SStream> streams;
    std::mutex mu;
    std::condition_variable cv;
    std::thread worker;
    bool stop = false;
    cudaStream_t s = nullptr;
    // per-round plan buffers (two slots)
    int64_t item_cap = 0;
    WorkItem *d_items[2] = {nullptr, nullptr};
    WorkItem *h_items[2] = {nullptr, nullptr};
    CUtensorMap *d_maps[2] = {nullptr, nullptr}, *h_maps[2] = {nullptr, nullptr};
    JobDesc *d_jobs[2] = {nullptr, nullptr}, *h_jobs[2] = {nullptr, nullptr};
    DecodeJob *d_dec[2] = {nullptr, nullptr}, *h_dec[2] = {nullptr, nullptr};  // blocks TMA cannot address
    CUtensorMap *d_dmaps[2] = {nullptr, nullptr}, *h_dmaps[2] = {nullptr, nullptr};  // TMA decode: 2 maps per block
    CUtensorMap *d_smaps[2] = {nullptr, nullptr}, *h_smaps[2] = {nullptr, nullptr};  // single pass: a map per block
    SmallScratch small;     // the N <= 256 single-pass kernel's scratch
    int single_force = 0;   // XENG_FUSED_KERNEL at creation
    DecTmaJob *d_djobs[2] = {nullptr, nullptr}, *h_djobs[2] = {nullptr, nullptr};
    SumJob *d_sjobs[2] = {nullptr, nullptr}, *h_sjobs[2] = {nullptr, nullptr};  // raw-nibble streams of a round
    int *d_err = nullptr, *h_err = nullptr;
    std::deque<Round> inflight;
    int next_slot = 0;
    std::vector<cudaEvent_t> free_events;
    // statistics
    std::vector<double> block_lat, dump_lat;
    double first_submit = -1, last_done = 0, ops_done = 0;
    int64_t rounds = 0, refused = 0, blocks_done = 0, dumps_done = 0, late_blocks = 0, short_dumps = 0;
    double gpu_decode_ms = 0, gpu_correlate_ms = 0, host_plan_ms = 0;
    std::vector<cudaEvent_t> free_timers;
    int sticky = XENG_OK;
};

namespace {

int64_t stream_bytes(const SStream &st, int max_blocks)
{
    const int64_t acc = (int64_t)st.F * n_baselines(st.N) * 8;
    if (st.single) return 3 * acc;  // accumulators and two dump buffers: its rounds read the blocks in place
    const int64_t planes = (int64_t)st.F * 2 * st.n_pad * (st.bs_pad * max_blocks);
    const int64_t part = (int64_t)st.F * (st.bs_pad * max_blocks / kTile) * st.n_pad * 8;
    const int64_t sums = (int64_t)st.F * st.n_pad * 8;
    // accumulators, two dump buffers, two plane slices with their nibble sums
    return 3 * acc + 2 * (planes + part + sums);
}

void free_stream_memory(SStream &st)
{
    cudaFree(st.acc);
    cudaFree(st.planes[0]);
    cudaFree(st.planes[1]);
    cudaFree(st.dump[0].buf);
    cudaFree(st.dump[1].buf);
    for (int k = 0; k < 2; k++) {
        cudaFree(st.partials[k]);
        cudaFree(st.sums[k]);
        st.partials[k] = nullptr;
        st.sums[k] = nullptr;
    }
    st.acc = nullptr;
    st.planes[0] = st.planes[1] = nullptr;
    st.dump[0].buf = st.dump[1].buf = nullptr;
}

double percentile(std::vector<double> v, double p)
{
    if (v.empty()) return 0;
    std::sort(v.begin(), v.end());
    const double x = p * (v.size() - 1);
    const size_t lo = (size_t)x;
    const size_t hi = std::min(v.size() - 1, lo + 1);
    return v[lo] + (v[hi] - v[lo]) * (x - lo);
}

// Publish finished rounds (caller holds `lk`).  If `wait_oldest`, first wait
// for the oldest round with the lock released, so submitters never wait on the GPU.
void reap(xserve_s *sv, std::unique_lock<std::mutex> &lk, bool wait_oldest)
{
    while (!sv->inflight.empty()) {
        cudaError_t q;
        if (wait_oldest) {
            cudaEvent_t ev = sv->inflight.front().ev;  // only this thread pops rounds
            lk.unlock();
            q = cudaEventSynchronize(ev);
            lk.lock();
            wait_oldest = false;
        } else {
            q = cudaEventQuery(sv->inflight.front().ev);
        }
        Round &r = sv->inflight.front();
        if (q == cudaErrorNotReady) break;
        if (q != cudaSuccess) {
            cudaGetLastError();
            sv->sticky = XENG_ERR_CUDA;
        }
        if (*(volatile int *)sv->h_err != 0) sv->sticky = XENG_ERR_TIMEOUT;
        const double t = now_s();
        for (auto &p : r.parts) {
            SStream &st = sv->streams[p.stream];
            for (double a : p.arrivals) sv->block_lat.push_back(t - a);
            st.consumed += p.nblocks;
            st.inflight -= p.nblocks;
            sv->blocks_done += p.nblocks;
            if (p.dump_slot >= 0) {
                DumpSlot &d = st.dump[p.dump_slot];
                d.ready = true;
                d.ready_time = t;
                sv->dump_lat.push_back(t - d.last_arrival);
                sv->dumps_done++;
                if (d.samples < st.dump_samples) sv->short_dumps++;
            }
        }
        sv->ops_done += r.useful_ops;
        sv->last_done = t;
        if (r.t0 && r.t1 && r.t2) {
            float a = 0, b = 0;
            if (cudaEventElapsedTime(&a, r.t0, r.t1) == cudaSuccess) sv->gpu_decode_ms += a;
            if (cudaEventElapsedTime(&b, r.t1, r.t2) == cudaSuccess) sv->gpu_correlate_ms += b;
            cudaGetLastError();
            sv->free_timers.push_back(r.t0);
            sv->free_timers.push_back(r.t1);
            sv->free_timers.push_back(r.t2);
        }
        sv->free_events.push_back(r.ev);
        sv->inflight.pop_front();
        sv->cv.notify_all();
    }
}

// Build and enqueue one round from the queued blocks (caller holds the lock).
// Returns false if nothing was ready.
cudaEvent_t take_timer(xserve_s *sv)
{
    if (!sv->free_timers.empty()) {
        cudaEvent_t e = sv->free_timers.back();
        sv->free_timers.pop_back();
        return e;
    }
    cudaEvent_t e = nullptr;
    if (cudaEventCreate(&e) != cudaSuccess) {
        cudaGetLastError();
        return nullptr;
    }
    return e;
}

bool launch_round(xserve_s *sv)
{
    const double host_t0 = now_s();
    const int slot = sv->next_slot;
    const int K = sv->opts.max_blocks;
    // nblocks == 0: the round only closes the stream's current integration
    // (its next queued block belongs to a later one, or a flush asked for it)
    struct Pick { int stream; int nblocks; };
    std::vector<Pick> picks;
    for (auto &st : sv->streams) {
        if (!st.open || st.queue.empty()) continue;
        const QBlock &head = st.queue.front();
        if (!head.ptr || head.integ > st.cur_integ) {
            if (st.integrated == 0) {
                // nothing of the current integration was integrated: move on without a dump
                st.cur_integ = head.ptr ? head.integ : std::max(st.cur_integ, head.integ + 1);
                if (!head.ptr) st.queue.pop_front();
                if (st.queue.empty() || !st.queue.front().ptr || st.queue.front().integ != st.cur_integ) continue;
            } else {
                if (st.dump[0].busy && st.dump[1].busy) continue;  // the close needs a free dump buffer
                picks.push_back({st.id, 0});
                continue;
            }
        }
        int nb = 0;
        for (const QBlock &qb : st.queue) {
            if (nb == K || !qb.ptr || qb.integ != st.cur_integ) break;
            ++nb;
        }
        const int64_t to_dump = (st.dump_samples - st.integrated) / st.block_samples;
        nb = (int)std::min<int64_t>(nb, to_dump);
        if (nb <= 0) continue;
        // the round that completes an integration needs a free dump buffer
        if (st.integrated + nb * st.block_samples == st.dump_samples && st.dump[0].busy && st.dump[1].busy) continue;
        picks.push_back({st.id, nb});
    }
    if (picks.empty()) return false;

    Round r;
    r.slot = slot;
    int64_t n_items = 0, n_dec = 0, dec_ctas = 0, n_djobs = 0, dtiles = 0, n_sjobs = 0, sum_entries = 0, n_smaps = 0;
    int jobi = 0;
    for (auto &pk : picks) {
        SStream &st = sv->streams[pk.stream];
        if (pk.nblocks == 0) {
            // close the integration short: its accumulators are final once the
            // rounds before this one complete, and this round does not touch them
            Round::Part part;
            part.stream = pk.stream;
            part.nblocks = 0;
            const int ds = st.dump[0].busy ? 1 : 0;
            DumpSlot &d = st.dump[ds];
            d.busy = true;
            d.ready = false;
            d.samples = st.integrated;
            d.blocks = st.integrated / st.block_samples;
            d.last_arrival = st.last_arrival;
            d.seq = st.cur_integ;
            part.dump_slot = ds;
            const QBlock &head = st.queue.front();
            st.cur_integ = head.ptr ? head.integ : std::max(st.cur_integ + 1, head.integ + 1);
            if (!head.ptr) st.queue.pop_front();
            st.integrated = 0;
            st.fresh = true;
            st.last_arrival = 0;
            r.parts.push_back(std::move(part));
            continue;
        }
        // a stream of the single-pass kernels: its blocks read where they are
        const int sk = st.single;
        if (sk) {
            Round::Part part;
            part.stream = pk.stream;
            part.nblocks = pk.nblocks;
            part.dump_slot = -1;
            Round::Single sg;
            sg.stream = pk.stream;
            sg.kernel = sk;
            sg.map0 = n_smaps;
            sg.nblocks = pk.nblocks;
            sg.store = st.fresh;
            for (int b = 0; b < pk.nblocks; b++) {
                QBlock qb = st.queue.front();
                st.queue.pop_front();
                part.arrivals.push_back(qb.arrival);
                st.last_arrival = std::max(st.last_arrival, qb.arrival);
                if (encode_single_pass_map(sk, sv->h_smaps[slot] + n_smaps++, qb.ptr, st.block_samples, st.F, st.N) !=
                    cudaSuccess) {
                    sv->sticky = XENG_ERR_CUDA;  // never launch with a descriptor that failed to encode
                    return false;
                }
            }
            r.singles.push_back(sg);
            r.useful_ops += 8.0 * (double)(pk.nblocks * st.block_samples) * st.F * (double)n_baselines(st.N);
            st.fresh = false;
            st.integrated += pk.nblocks * st.block_samples;
            st.inflight += pk.nblocks;
            if (st.integrated == st.dump_samples) {
                const int ds = st.dump[0].busy ? 1 : 0;
                DumpSlot &d = st.dump[ds];
                d.busy = true;
                d.ready = false;
                d.samples = st.integrated;
                d.blocks = st.integrated / st.block_samples;
                d.last_arrival = st.last_arrival;
                d.seq = st.cur_integ++;
                part.dump_slot = ds;
                st.integrated = 0;
                st.fresh = true;
                st.last_arrival = 0;
            }
            r.parts.push_back(std::move(part));
            continue;
        }
        const int64_t pitch = st.bs_pad * pk.nblocks;
        uint8_t *pl = st.planes[slot];
        // raw-nibble planes when every block of the round goes through the TMA
        // decode and the round spans at most kFusedMaxSamples samples
        bool raw = st.partials[slot] && pitch <= kFusedMaxSamples;
        for (int b = 0; raw && b < pk.nblocks; b++) raw = decode_tma_ok(st.queue[b].ptr, st.N);
        Round::Part part;
        part.stream = pk.stream;
        part.nblocks = pk.nblocks;
        part.dump_slot = -1;
        for (int b = 0; b < pk.nblocks; b++) {
            QBlock qb = st.queue.front();
            st.queue.pop_front();
            part.arrivals.push_back(qb.arrival);
            st.last_arrival = std::max(st.last_arrival, qb.arrival);
            // the TMA decode where the block's rows allow it: the block's raw
            // map and the slice's plane map, the block at column b * bs_pad
            CUtensorMap *mp = sv->h_dmaps[slot] + 2 * n_djobs;
            const bool tma = encode_decode_tma_maps(qb.ptr, st.block_samples, st.F, st.N, pl, pitch, st.n_pad, mp,
                                                    mp + 1);
            if (raw && !tma) {
                sv->sticky = XENG_ERR_CUDA;  // a block checked above could not be encoded
                return false;
            }
            if (tma) {
                DecTmaJob &dt = sv->h_djobs[slot][n_djobs++];
                dt.tile0 = dtiles;
                dt.T = st.block_samples;
                dt.n_ib = (int32_t)(st.n_pad / kTile);
                dt.n_tb = (int32_t)(st.bs_pad / kTile);
                dt.F = st.F;
                dt.N = st.N;
                dt.n_pad = (int32_t)st.n_pad;
                dt.x0 = (int32_t)(b * st.bs_pad);
                dt.partials = raw ? st.partials[slot] : nullptr;
                dt.part_n_tb = (int32_t)(pitch / kTile);
                dt.pad_ = 0;
                dtiles += (int64_t)dt.n_ib * dt.F * dt.n_tb;
            } else {
                DecodeJob &dj = sv->h_dec[slot][n_dec++];
                dj.block = qb.ptr;
                dj.planes = pl + b * st.bs_pad;
                dj.T = st.block_samples;
                dj.t_pad = st.bs_pad;
                dj.pitch = pitch;
                dj.n_pad = st.n_pad;
                dj.cta0 = dec_ctas;
                dj.F = st.F;
                dj.N = st.N;
                dj.vec_ok = decode_vec_ok(qb.ptr, st.N);
                dj.pad_ = 0;
                dec_ctas += decode_ctas(st.bs_pad, st.n_pad, st.F);
            }
        }
        if (encode_planes_map(&sv->h_maps[slot][jobi], pl, pitch, (int64_t)st.F * 2 * st.n_pad) != cudaSuccess) {
            sv->sticky = XENG_ERR_CUDA;  // never launch with a descriptor that failed to encode
            return false;
        }
        JobDesc &jd = sv->h_jobs[slot][jobi];
        jd.out = st.acc;
        jd.n_pad = (int32_t)st.n_pad;
        jd.N = st.N;
        jd.mode = st.fresh ? 0 : 1;
        jd.n_samples = (int32_t)(pk.nblocks * st.block_samples);
        jd.sums = raw ? st.sums[slot] : nullptr;
        if (raw) {
            SumJob &sj = sv->h_sjobs[slot][n_sjobs++];
            sj.partials = st.partials[slot];
            sj.sums = st.sums[slot];
            sj.first = sum_entries;
            sj.n_tb = (int32_t)(pitch / kTile);
            sj.part_n_tb = (int32_t)(pitch / kTile);
            sj.n_pad = (int32_t)st.n_pad;
            sj.pad_ = 0;
            sum_entries += (int64_t)st.F * st.n_pad;
        }
        const int nt = (int)(st.n_pad / kTile);
        const int n_k = (int)(pitch / kTile);
        for (int f = 0; f < st.F; f++)
            for (int I = 0; I < nt; I++)
                for (int J = I; J < nt; J++) {
                    WorkItem &w = sv->h_items[slot][n_items++];
                    w.job = jobi;
                    w.fl = f;
                    w.I = (int16_t)I;
                    w.J = (int16_t)J;
                    w.kc0 = 0;
                    w.kc1 = n_k;
                }
        r.useful_ops += 8.0 * (double)(pk.nblocks * st.block_samples) * st.F * (double)n_baselines(st.N);
        st.fresh = false;
        st.integrated += pk.nblocks * st.block_samples;
        st.inflight += pk.nblocks;
        if (st.integrated == st.dump_samples) {
            const int ds = st.dump[0].busy ? 1 : 0;
            DumpSlot &d = st.dump[ds];
            d.busy = true;
            d.ready = false;
            d.samples = st.integrated;
            d.blocks = st.integrated / st.block_samples;
            d.last_arrival = st.last_arrival;
            d.seq = st.cur_integ++;
            part.dump_slot = ds;
            st.integrated = 0;
            st.fresh = true;
            st.last_arrival = 0;
        }
        r.parts.push_back(std::move(part));
        ++jobi;
    }

    cudaStream_t s = sv->s;
    r.t0 = take_timer(sv);
    r.t1 = take_timer(sv);
    r.t2 = take_timer(sv);
    cudaError_t e = cudaSuccess;
    if (n_dec > 0) e = cudaMemcpyAsync(sv->d_dec[slot], sv->h_dec[slot], n_dec * sizeof(DecodeJob), cudaMemcpyHostToDevice, s);
    if (e == cudaSuccess && n_djobs > 0)
        e = cudaMemcpyAsync(sv->d_dmaps[slot], sv->h_dmaps[slot], 2 * n_djobs * sizeof(CUtensorMap), cudaMemcpyHostToDevice,
                            s);
    if (e == cudaSuccess && n_djobs > 0)
        e = cudaMemcpyAsync(sv->d_djobs[slot], sv->h_djobs[slot], n_djobs * sizeof(DecTmaJob), cudaMemcpyHostToDevice, s);
    if (e == cudaSuccess && n_sjobs > 0)
        e = cudaMemcpyAsync(sv->d_sjobs[slot], sv->h_sjobs[slot], n_sjobs * sizeof(SumJob), cudaMemcpyHostToDevice, s);
    if (e == cudaSuccess && jobi > 0)
        e = cudaMemcpyAsync(sv->d_maps[slot], sv->h_maps[slot], jobi * sizeof(CUtensorMap), cudaMemcpyHostToDevice, s);
    if (e == cudaSuccess && jobi > 0)
        e = cudaMemcpyAsync(sv->d_jobs[slot], sv->h_jobs[slot], jobi * sizeof(JobDesc), cudaMemcpyHostToDevice, s);
    if (e == cudaSuccess && n_items > 0)
        e = cudaMemcpyAsync(sv->d_items[slot], sv->h_items[slot], n_items * sizeof(WorkItem), cudaMemcpyHostToDevice, s);
    if (e == cudaSuccess && n_smaps > 0)
        e = cudaMemcpyAsync(sv->d_smaps[slot], sv->h_smaps[slot], n_smaps * sizeof(CUtensorMap), cudaMemcpyHostToDevice,
                            s);
    if (e == cudaSuccess && r.t0) e = cudaEventRecord(r.t0, s);
    if (e == cudaSuccess)
        e = launch_decode_tma_batch(sv->d_dmaps[slot], sv->d_djobs[slot], (int)n_djobs, dtiles, sv->d_err, sv->num_sms, s);
    if (e == cudaSuccess && n_dec > 0) e = launch_decode_batch(sv->d_dec[slot], (int)n_dec, dec_ctas, s);
    if (e == cudaSuccess && n_sjobs > 0)
        e = launch_plane_sums_batch(sv->d_sjobs[slot], (int32_t)n_sjobs, sum_entries, sv->num_sms, s);
    if (e == cudaSuccess && r.t1) e = cudaEventRecord(r.t1, s);
    if (e == cudaSuccess && n_items > 0) {
        ListArgs L;
        L.maps = sv->d_maps[slot];
        L.jobs = sv->d_jobs[slot];
        L.items = sv->d_items[slot];
        L.cta_begin = nullptr;  // round-robin over the items
        L.err = sv->d_err;
        L.n_items = n_items;
        e = launch_correlate_tc_listed(L, (int)std::min<int64_t>(sv->num_sms, n_items), s);
    }
    for (const auto &sg : r.singles) {
        // launches of at most kFusedMaxSamples samples (whole blocks), the first
        // storing when the round opens an integration
        const SStream &st = sv->streams[sg.stream];
        const int per = (int)(kFusedMaxSamples / st.block_samples);
        const int spb = (int)(st.block_samples / single_pass_stage(sg.kernel));
        for (int b0 = 0; b0 < sg.nblocks && e == cudaSuccess; b0 += per) {
            const int nb = std::min(per, sg.nblocks - b0);
            const int64_t nt = (int64_t)nb * st.block_samples;
            e = launch_single_pass(sg.kernel, nullptr, nt, 0, nt, st.F, st.N, 0, st.F, st.acc,
                                   (sg.store && b0 == 0) ? 0 : 1, &sv->small, sv->d_err, sv->num_sms, s,
                                   sv->d_smaps[slot] + sg.map0 + b0, spb);
        }
    }
    if (e == cudaSuccess && r.t2) e = cudaEventRecord(r.t2, s);
    for (auto &p : r.parts) {
        if (p.dump_slot < 0 || e != cudaSuccess) continue;
        SStream &st = sv->streams[p.stream];
        e = cudaMemcpyAsync(st.dump[p.dump_slot].buf, st.acc, (size_t)st.F * n_baselines(st.N) * 8,
                            cudaMemcpyDeviceToDevice, s);
    }
    if (e == cudaSuccess) e = cudaMemcpyAsync(sv->h_err, sv->d_err, sizeof(int), cudaMemcpyDeviceToHost, s);
    if (!sv->free_events.empty()) {
        r.ev = sv->free_events.back();
        sv->free_events.pop_back();
    } else if (e == cudaSuccess) {
        e = cudaEventCreateWithFlags(&r.ev, cudaEventDisableTiming);
    }
    if (e == cudaSuccess) e = cudaEventRecord(r.ev, s);
    if (e != cudaSuccess) {
        cudaGetLastError();
        sv->sticky = XENG_ERR_CUDA;
        return false;
    }
    sv->inflight.push_back(std::move(r));
    sv->next_slot ^= 1;
    sv->rounds++;
    sv->host_plan_ms += (now_s() - host_t0) * 1e3;
    return true;
}

void worker_main(xserve_s *sv)
{
    cudaSetDevice(sv->device);
    std::unique_lock<std::mutex> lk(sv->mu);
    while (true) {
        reap(sv, lk, false);
        if (sv->stop) {
            bool busy = !sv->inflight.empty();
            for (auto &st : sv->streams) busy = busy || (st.open && !st.queue.empty());
            if (!busy || sv->sticky != XENG_OK) break;
        }
        if (sv->sticky != XENG_OK) {
            sv->cv.wait_for(lk, std::chrono::milliseconds(5));
            continue;
        }
        if (sv->inflight.size() >= 2) {
            // the slot about to be reused must be free: wait for the oldest round
            reap(sv, lk, true);
            continue;
        }
        if (launch_round(sv)) continue;
        if (!sv->inflight.empty()) {
            lk.unlock();
            std::this_thread::sleep_for(std::chrono::microseconds(20));
            lk.lock();
        } else {
            sv->cv.wait_for(lk, std::chrono::milliseconds(2));
        }
    }
    while (!sv->inflight.empty()) reap(sv, lk, true);
}

}  // namespace

extern "C" {

double xserve_now(void) { return now_s(); }

int xserve_create(const xserve_opts_t *opts, xserve_t *out)
{
    if (!out) return XENG_ERR_ARG;
    int dev = 0, major = 0, minor = 0, sms = 0;
    if (cudaGetDevice(&dev) != cudaSuccess ||
        cudaDeviceGetAttribute(&major, cudaDevAttrComputeCapabilityMajor, dev) != cudaSuccess ||
        cudaDeviceGetAttribute(&minor, cudaDevAttrComputeCapabilityMinor, dev) != cudaSuccess ||
        cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess) {
        cudaGetLastError();
        return XENG_ERR_UNSUPPORTED;
    }
    if (major != 10 || minor != 3) return XENG_ERR_UNSUPPORTED;
    xserve_opts_t o;
    o.hbm_budget_bytes = (int64_t)120 << 30;
    o.max_blocks = 16;
    o.max_streams = 16;
    o.max_items = 4 << 20;
    o.compute_budget_tops = 0;
    if (opts) o = *opts;
    if (o.hbm_budget_bytes <= 0 || o.max_blocks < 1 || o.max_streams < 1 || o.max_items < 1 || o.max_streams > 4096)
        return XENG_ERR_RANGE;
    xserve_s *sv = new (std::nothrow) xserve_s;
    if (!sv) return XENG_ERR_NOMEM;
    sv->opts = o;
    sv->device = dev;
    sv->num_sms = sms;
    sv->streams.resize(o.max_streams);
    for (int k = 0; k < o.max_streams; k++) sv->streams[k].id = k;
    cudaError_t e = prepare_correlate_tc_listed();
    if (e == cudaSuccess) e = prepare_decode_tma_batch();
    if (e == cudaSuccess) e = cudaStreamCreateWithFlags(&sv->s, cudaStreamNonBlocking);
    for (int k = 0; k < 2 && e == cudaSuccess; k++) {
        e = cudaMalloc(&sv->d_items[k], (size_t)o.max_items * sizeof(WorkItem));
        if (e == cudaSuccess) e = cudaMallocHost(&sv->h_items[k], (size_t)o.max_items * sizeof(WorkItem));
        if (e == cudaSuccess) e = cudaMalloc(&sv->d_maps[k], (size_t)o.max_streams * sizeof(CUtensorMap));
        if (e == cudaSuccess) e = cudaMallocHost(&sv->h_maps[k], (size_t)o.max_streams * sizeof(CUtensorMap));
        if (e == cudaSuccess) e = cudaMalloc(&sv->d_jobs[k], (size_t)o.max_streams * sizeof(JobDesc));
        if (e == cudaSuccess) e = cudaMallocHost(&sv->h_jobs[k], (size_t)o.max_streams * sizeof(JobDesc));
        if (e == cudaSuccess) e = cudaMalloc(&sv->d_dec[k], (size_t)o.max_streams * o.max_blocks * sizeof(DecodeJob));
        if (e == cudaSuccess) e = cudaMallocHost(&sv->h_dec[k], (size_t)o.max_streams * o.max_blocks * sizeof(DecodeJob));
        if (e == cudaSuccess)
            e = cudaMalloc(&sv->d_dmaps[k], (size_t)o.max_streams * o.max_blocks * 2 * sizeof(CUtensorMap));
        if (e == cudaSuccess)
            e = cudaMallocHost(&sv->h_dmaps[k], (size_t)o.max_streams * o.max_blocks * 2 * sizeof(CUtensorMap));
        if (e == cudaSuccess) e = cudaMalloc(&sv->d_djobs[k], (size_t)o.max_streams * o.max_blocks * sizeof(DecTmaJob));
        if (e == cudaSuccess)
            e = cudaMallocHost(&sv->h_djobs[k], (size_t)o.max_streams * o.max_blocks * sizeof(DecTmaJob));
        if (e == cudaSuccess) e = cudaMalloc(&sv->d_sjobs[k], (size_t)o.max_streams * sizeof(SumJob));
        if (e == cudaSuccess) e = cudaMallocHost(&sv->h_sjobs[k], (size_t)o.max_streams * sizeof(SumJob));
        if (e == cudaSuccess) e = cudaMalloc(&sv->d_smaps[k], (size_t)o.max_streams * o.max_blocks * sizeof(CUtensorMap));
        if (e == cudaSuccess)
            e = cudaMallocHost(&sv->h_smaps[k], (size_t)o.max_streams * o.max_blocks * sizeof(CUtensorMap));
    }
    sv->single_force = single_pass_force_from_env();
    if (e == cudaSuccess) e = cudaMalloc(&sv->d_err, sizeof(int));
    if (e == cudaSuccess) e = cudaMemset(sv->d_err, 0, sizeof(int));
    if (e == cudaSuccess) e = cudaMallocHost(&sv->h_err, sizeof(int));
    if (e != cudaSuccess) {
        cudaGetLastError();
        xserve_destroy(sv);
        return e == cudaErrorMemoryAllocation ? XENG_ERR_NOMEM : XENG_ERR_CUDA;
    }
    *sv->h_err = 0;
    sv->worker = std::thread(worker_main, sv);
    *out = sv;
    return XENG_OK;
}

int xserve_open_stream(xserve_t sv, int32_t n_inputs, int32_t n_freq, int64_t block_samples, int64_t dump_samples,
                       double rate_blocks_per_s, int32_t *stream_id)
{
    if (!sv || !stream_id) return XENG_ERR_ARG;
    if (n_inputs < 1 || n_inputs > XENG_MAX_INPUTS || n_freq < 1 || block_samples < 1 || dump_samples < block_samples ||
        dump_samples % block_samples != 0 || dump_samples > XENG_MAX_T_INTEG || rate_blocks_per_s < 0)
        return XENG_ERR_RANGE;
    const int64_t bs_pad = round_up(block_samples, kTile);
    if (bs_pad * sv->opts.max_blocks > kMaxChunkSamples) return XENG_ERR_RANGE;  // one round stays exact in f32
    const int64_t n_pad = round_up(n_inputs, kTile);
    const int64_t items = (int64_t)n_freq * (n_pad / kTile) * (n_pad / kTile + 1) / 2;
    std::unique_lock<std::mutex> lk(sv->mu);
    int64_t items_open = 0;
    int free_id = -1;
    for (auto &st : sv->streams) {
        if (st.open) items_open += (int64_t)st.F * (st.n_pad / kTile) * (st.n_pad / kTile + 1) / 2;
        else if (free_id < 0) free_id = st.id;
    }
    if (free_id < 0 || items_open + items > sv->opts.max_items) {
        sv->refused++;
        return XENG_ERR_NOMEM;
    }
    SStream probe;
    probe.N = n_inputs;
    probe.F = n_freq;
    probe.n_pad = n_pad;
    probe.bs_pad = bs_pad;
    // a shape a single-pass kernel takes (blocks a whole number of its stages, at
    // most a launch's samples; 16-byte aligned blocks are then required)
    if (block_samples <= kFusedMaxSamples) {
        const int k = single_pass_kernel(nullptr, n_inputs, sv->single_force, true);
        if (k && block_samples % single_pass_stage(k) == 0) probe.single = k;
    }
    const int64_t bytes = stream_bytes(probe, sv->opts.max_blocks);
    const double demand = rate_blocks_per_s * 8.0 * block_samples * n_freq * (double)n_baselines(n_inputs) / 1e12;
    if (sv->used_bytes + bytes > sv->opts.hbm_budget_bytes ||
        (sv->opts.compute_budget_tops > 0 && sv->used_tops + demand > sv->opts.compute_budget_tops)) {
        sv->refused++;
        return XENG_ERR_NOMEM;  // admission refused: over the HBM (or compute) budget
    }
    SStream &st = sv->streams[free_id];
    st = SStream();
    st.id = free_id;
    st.N = n_inputs;
    st.F = n_freq;
    st.block_samples = block_samples;
    st.bs_pad = bs_pad;
    st.dump_samples = dump_samples;
    st.n_pad = n_pad;
    st.single = probe.single;
    st.demand_tops = demand;
    st.bytes = bytes;
    st.seen.assign((size_t)(dump_samples / block_samples), 0);
    const size_t acc = (size_t)n_freq * n_baselines(n_inputs) * 8;
    const size_t planes = (size_t)n_freq * 2 * n_pad * bs_pad * sv->opts.max_blocks;
    cudaError_t e = cudaMalloc(&st.acc, acc);
    if (e == cudaSuccess) e = cudaMalloc(&st.dump[0].buf, acc);
    if (e == cudaSuccess) e = cudaMalloc(&st.dump[1].buf, acc);
    if (e == cudaSuccess && !st.single) e = cudaMalloc(&st.planes[0], planes);
    if (e == cudaSuccess && !st.single) e = cudaMalloc(&st.planes[1], planes);
    const size_t part = (size_t)n_freq * (bs_pad * sv->opts.max_blocks / kTile) * n_pad * sizeof(int2);
    const size_t sums = (size_t)n_freq * n_pad * sizeof(int2);
    for (int k = 0; k < 2 && e == cudaSuccess && !st.single; k++) {
        e = cudaMalloc(&st.partials[k], part);
        if (e == cudaSuccess) e = cudaMalloc(&st.sums[k], sums);
    }
    if (e != cudaSuccess) {
        cudaGetLastError();
        free_stream_memory(st);
        sv->refused++;
        return XENG_ERR_NOMEM;
    }
    st.open = true;
    sv->used_bytes += bytes;
    sv->used_tops += demand;
    *stream_id = free_id;
    return XENG_OK;
}

namespace {

// Queue block number `seq` of the stream (caller holds the lock).
int submit_locked(xserve_s *sv, SStream &st, const uint8_t *block, int64_t seq, double t)
{
    if (st.single && (reinterpret_cast<uintptr_t>(block) & 15) != 0) return XENG_ERR_ARG;  // read by TMA in place
    const int64_t bpd = st.blocks_per_dump();
    const int64_t integ = seq / bpd;
    if (integ < st.top_integ) {  // a later integration's block has closed this one
        sv->late_blocks++;
        return XENG_ERR_LATE;
    }
    if (integ > st.top_integ) {
        st.top_integ = integ;
        std::fill(st.seen.begin(), st.seen.end(), 0);
    }
    uint8_t &seen = st.seen[(size_t)(seq - integ * bpd)];
    if (seen) return XENG_ERR_ARG;  // this block number was submitted already
    seen = 1;
    st.queue.push_back({block, t, integ});
    st.submitted++;
    st.next_block = std::max(st.next_block, seq + 1);
    if (sv->first_submit < 0 || t < sv->first_submit) sv->first_submit = t;
    sv->cv.notify_all();
    return XENG_OK;
}

}  // namespace

int xserve_submit(xserve_t sv, int32_t stream_id, const uint8_t *block, double arrival_s)
{
    if (!sv || !block) return XENG_ERR_ARG;
    const double t = arrival_s > 0 ? arrival_s : now_s();  // stamped before any wait for the lock
    std::unique_lock<std::mutex> lk(sv->mu);
    if (stream_id < 0 || stream_id >= (int)sv->streams.size() || !sv->streams[stream_id].open) return XENG_ERR_ARG;
    if (sv->sticky != XENG_OK) return sv->sticky;
    SStream &st = sv->streams[stream_id];
    return submit_locked(sv, st, block, st.next_block, t);
}

int xserve_submit_seq(xserve_t sv, int32_t stream_id, const uint8_t *block, int64_t seq, double arrival_s)
{
    if (!sv || !block || seq < 0) return XENG_ERR_ARG;
    const double t = arrival_s > 0 ? arrival_s : now_s();
    std::unique_lock<std::mutex> lk(sv->mu);
    if (stream_id < 0 || stream_id >= (int)sv->streams.size() || !sv->streams[stream_id].open) return XENG_ERR_ARG;
    if (sv->sticky != XENG_OK) return sv->sticky;
    return submit_locked(sv, sv->streams[stream_id], block, seq, t);
}

int xserve_flush(xserve_t sv, int32_t stream_id)
{
    if (!sv) return XENG_ERR_ARG;
    std::unique_lock<std::mutex> lk(sv->mu);
    if (stream_id < 0 || stream_id >= (int)sv->streams.size() || !sv->streams[stream_id].open) return XENG_ERR_ARG;
    if (sv->sticky != XENG_OK) return sv->sticky;
    SStream &st = sv->streams[stream_id];
    // later blocks belong to the next integration
    st.queue.push_back({nullptr, 0.0, st.top_integ});
    st.top_integ++;
    std::fill(st.seen.begin(), st.seen.end(), 0);
    st.next_block = std::max(st.next_block, st.top_integ * st.blocks_per_dump());
    sv->cv.notify_all();
    return XENG_OK;
}

int64_t xserve_consumed(xserve_t sv, int32_t stream_id)
{
    if (!sv) return XENG_ERR_ARG;
    std::unique_lock<std::mutex> lk(sv->mu);
    if (stream_id < 0 || stream_id >= (int)sv->streams.size() || !sv->streams[stream_id].open) return XENG_ERR_ARG;
    return sv->streams[stream_id].consumed;
}

int xserve_poll_dump(xserve_t sv, int32_t stream_id, int32_t *out, xserve_dump_info_t *info)
{
    if (!sv || !out) return XENG_ERR_ARG;
    std::unique_lock<std::mutex> lk(sv->mu);
    if (stream_id < 0 || stream_id >= (int)sv->streams.size() || !sv->streams[stream_id].open) return XENG_ERR_ARG;
    SStream &st = sv->streams[stream_id];
    int pick = -1;
    for (int k = 0; k < 2; k++)
        if (st.dump[k].busy && st.dump[k].ready && (pick < 0 || st.dump[k].seq < st.dump[pick].seq)) pick = k;
    if (pick < 0) return sv->sticky != XENG_OK ? sv->sticky : 0;
    DumpSlot &d = st.dump[pick];
    const size_t bytes = (size_t)st.F * n_baselines(st.N) * 8;
    lk.unlock();
    cudaError_t e = cudaMemcpy(out, d.buf, bytes, cudaMemcpyDefault);  // the copy into d.buf has completed
    lk.lock();
    if (e != cudaSuccess) {
        cudaGetLastError();
        return XENG_ERR_CUDA;
    }
    if (info) {
        info->seq = d.seq;
        info->samples = d.samples;
        info->last_arrival_s = d.last_arrival;
        info->ready_s = d.ready_time;
        info->blocks = d.blocks;
        info->missing_blocks = st.blocks_per_dump() - d.blocks;
    }
    d.busy = false;
    d.ready = false;
    sv->cv.notify_all();
    return 1;
}

int xserve_drain(xserve_t sv, double timeout_s)
{
    if (!sv) return XENG_ERR_ARG;
    std::unique_lock<std::mutex> lk(sv->mu);
    const double t_end = now_s() + (timeout_s > 0 ? timeout_s : 1e9);
    while (true) {
        bool busy = !sv->inflight.empty();
        for (auto &st : sv->streams) {
            if (!st.open || st.queue.empty()) continue;
            // a stream whose next round waits for the client to take a dump does not count
            const QBlock &head = st.queue.front();
            const bool closes = !head.ptr || head.integ > st.cur_integ;
            const bool blocked = st.dump[0].busy && st.dump[1].busy &&
                                 ((closes && st.integrated > 0) ||
                                  st.integrated + st.block_samples * std::min<int64_t>(sv->opts.max_blocks, st.queue.size()) >=
                                      st.dump_samples);
            busy = busy || !blocked;
        }
        if (!busy || sv->sticky != XENG_OK) break;
        if (now_s() > t_end) return XENG_ERR_TIMEOUT;
        sv->cv.wait_for(lk, std::chrono::milliseconds(1));
    }
    return sv->sticky;
}

int xserve_close_stream(xserve_t sv, int32_t stream_id)
{
    if (!sv) return XENG_ERR_ARG;
    std::unique_lock<std::mutex> lk(sv->mu);
    if (stream_id < 0 || stream_id >= (int)sv->streams.size() || !sv->streams[stream_id].open) return XENG_ERR_ARG;
    SStream &st = sv->streams[stream_id];
    st.queue.clear();  // blocks never launched are dropped
    while (st.inflight > 0 && sv->sticky == XENG_OK) sv->cv.wait_for(lk, std::chrono::milliseconds(1));
    st.open = false;
    sv->used_bytes -= st.bytes;
    sv->used_tops -= st.demand_tops;
    free_stream_memory(st);
    return XENG_OK;
}

int xserve_stats(xserve_t sv, xserve_stats_t *out)
{
    if (!sv || !out) return XENG_ERR_ARG;
    std::unique_lock<std::mutex> lk(sv->mu);
    memset(out, 0, sizeof(*out));
    out->rounds = sv->rounds;
    out->blocks_done = sv->blocks_done;
    out->dumps_done = sv->dumps_done;
    out->refused = sv->refused;
    int64_t backlog = 0;
    int open = 0;
    for (auto &st : sv->streams) {
        if (!st.open) continue;
        ++open;
        for (const QBlock &qb : st.queue) backlog += qb.ptr ? 1 : 0;
    }
    out->open_streams = open;
    out->backlog_blocks = backlog;
    out->used_bytes = sv->used_bytes;
    out->useful_ops = sv->ops_done;
    out->busy_s = sv->first_submit >= 0 ? sv->last_done - sv->first_submit : 0;
    out->block_p50_s = percentile(sv->block_lat, 0.50);
    out->block_p99_s = percentile(sv->block_lat, 0.99);
    out->dump_p50_s = percentile(sv->dump_lat, 0.50);
    out->dump_p99_s = percentile(sv->dump_lat, 0.99);
    out->gpu_decode_ms = sv->gpu_decode_ms;
    out->gpu_correlate_ms = sv->gpu_correlate_ms;
    out->host_plan_ms = sv->host_plan_ms;
    out->late_blocks = sv->late_blocks;
    out->short_dumps = sv->short_dumps;
    return sv->sticky;
}

void xserve_destroy(xserve_t sv)
{
    if (!sv) return;
    {
        std::unique_lock<std::mutex> lk(sv->mu);
        sv->stop = true;
        for (auto &st : sv->streams) st.queue.clear();
        sv->cv.notify_all();
    }
    if (sv->worker.joinable()) sv->worker.join();
    cudaDeviceSynchronize();
    for (auto &st : sv->streams) free_stream_memory(st);
    for (int k = 0; k < 2; k++) {
        cudaFree(sv->d_items[k]);
        cudaFreeHost(sv->h_items[k]);
        cudaFree(sv->d_maps[k]);
        cudaFreeHost(sv->h_maps[k]);
        cudaFree(sv->d_jobs[k]);
        cudaFreeHost(sv->h_jobs[k]);
        cudaFree(sv->d_dec[k]);
        cudaFreeHost(sv->h_dec[k]);
        cudaFree(sv->d_dmaps[k]);
        cudaFreeHost(sv->h_dmaps[k]);
        cudaFree(sv->d_djobs[k]);
        cudaFreeHost(sv->h_djobs[k]);
        cudaFree(sv->d_sjobs[k]);
        cudaFreeHost(sv->h_sjobs[k]);
        cudaFree(sv->d_smaps[k]);
        cudaFreeHost(sv->h_smaps[k]);
    }
    small_scratch_free(&sv->small);
    cudaFree(sv->d_err);
    if (sv->h_err) cudaFreeHost(sv->h_err);
    for (auto e : sv->free_events) cudaEventDestroy(e);
    for (auto e : sv->free_timers) cudaEventDestroy(e);
    if (sv->s) cudaStreamDestroy(sv->s);
    cudaGetLastError();
    delete sv;
}

}  // extern "C"
