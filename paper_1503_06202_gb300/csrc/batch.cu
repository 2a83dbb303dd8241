// batch.cu -- many independent correlations (uneven N, F, T) in one pass:
// one persistent TMA decode launch over every job's tiles (plus a
// thread-per-row decode launch for jobs whose rows TMA cannot address), then
// one persistent tensor-core launch over a host-planned work list, all
// captured once in a CUDA graph and replayed per run.  Each job is a whole integration (paper Sec. IV-C-1)
// written to its own output; results are bit-identical to correlating each
// job alone.
//
// Planning: every job gets its own region of one decode buffer and its own
// TMA descriptor.  Jobs the TMA decode can address get raw-nibble planes (E4M3
// codes of u / 512, as the single-instance path): the decode also writes each
// tile's per-input nibble sums, one small launch totals them per job, and the
// correlation's epilogue applies the offset terms (their items then span at
// most 32,768 samples, keeping every f32 sum below 2^24).  Its upper-triangle 128x128 tile pairs (per channel) become
// work items; a tile whose integration is longer than `max_chunks` 128-sample
// chunks is split along time into several items whose int32 results are added
// with atomics (exact: integer addition is order-independent).  Items are
// assigned to one persistent CTA per SM longest-first onto the least-loaded
// CTA (LPT), round-robin in job order, or in job order onto the CTA expected
// to be free first (ORDERED: the CTAs move through the list together and share
// each channel's operands in L2); each CTA runs its items in job/channel order,
// a channel's tiles row by row, by diagonal or in Z (Morton) order.
//
// Jobs a single-pass kernel takes (N a multiple of 16 up to the build's bound,
// block 16-byte aligned: the kernel a handle would run for that N) skip the
// planes and run in the same graph -- no decode traffic, and no host call,
// checks or launch gap between jobs.  Those of the 2-CTA pair kernel with at
// most 32,768 samples share one persistent launch over all their block pairs
// (jobs longest first, so the round-robin over the clusters stays balanced and
// no job leaves the GPU half idle at its end); the others get single-pass
// launches of up to 32,768 samples each.  The environment variable
// XENG_FUSED_KERNEL (read at creation) forces a kernel for them as for a
// handle; "none" sends every job through the planes.
#include <algorithm>
#include <cinttypes>
#include <cstdio>
#include <cstring>
#include <new>
#include <queue>
#include <string>
#include <vector>

#include "../../include/xeng.h"
#include "xeng_internal.h"

using namespace xeng;

struct xeng_batch_s {
    std::vector<xeng_job_t> jobs;
    xeng_batch_opts_t opts{};
    int device = 0, num_sms = 0;
    uint8_t *planes = nullptr;
    int64_t planes_bytes = 0;
    CUtensorMap *d_maps = nullptr;
    JobDesc *d_jobs = nullptr;
    WorkItem *d_items = nullptr;
    int32_t *d_cta_begin = nullptr;
    DecodeJob *d_dec = nullptr;    // jobs whose rows TMA cannot address: thread-per-row decode
    int n_dec = 0;
    int64_t dec_ctas = 0;
    CUtensorMap *d_dmaps = nullptr;  // the other jobs: TMA decode (raw map, plane map per job)
    DecTmaJob *d_djobs = nullptr;
    int n_djobs = 0;
    int64_t dtiles = 0;
    int2 *partials = nullptr;        // raw-nibble jobs: per-tile nibble sums, then their totals
    int2 *sums = nullptr;
    SumJob *d_sjobs = nullptr;
    int n_sjobs = 0;
    int64_t sum_entries = 0;
    std::vector<std::pair<int, int>> single;  // (job, single-pass kernel) in job order
    std::vector<char> listed;                   // per job: in the pair kernel's listed launch
    PairJob *d_pjobs = nullptr;                 // that launch's jobs and their maps
    CUtensorMap *d_pmaps = nullptr;
    int n_pjobs = 0;
    int64_t p_items = 0;
    SmallScratch small;                         // the N <= 256 kernel's scratch, if a job takes it
    int grid = 0;
    int64_t n_items = 0;
    double max_load = 0, mean_load = 0;
    std::vector<std::pair<int32_t *, size_t>> zero_outs;  // outputs of split jobs, cleared each run
    int *d_err = nullptr, *h_err = nullptr;
    cudaStream_t cap = nullptr;
    cudaStream_t side = nullptr;     // second branch of a run: the N <= 256 kernel's jobs
    cudaEvent_t fork = nullptr, join = nullptr;
    cudaGraph_t graph = nullptr;
    cudaGraphExec_t exec = nullptr;
    int sticky = XENG_OK;
};

namespace {

int status_of(cudaError_t e)
{
    if (e == cudaSuccess) return XENG_OK;
    cudaGetLastError();
    return e == cudaErrorMemoryAllocation ? XENG_ERR_NOMEM : XENG_ERR_CUDA;
}

bool on_device(const void *p)
{
    cudaPointerAttributes at;
    if (cudaPointerGetAttributes(&at, p) != cudaSuccess) {
        cudaGetLastError();
        return false;
    }
    return at.type == cudaMemoryTypeDevice || at.type == cudaMemoryTypeManaged;
}

template <class T>
cudaError_t upload(T **dst, const std::vector<T> &v)
{
    const size_t bytes = std::max<size_t>(v.size(), 1) * sizeof(T);
    cudaError_t e = cudaMalloc(dst, bytes);
    if (e == cudaSuccess && !v.empty()) e = cudaMemcpy(*dst, v.data(), v.size() * sizeof(T), cudaMemcpyHostToDevice);
    return e;
}

void free_batch(xeng_batch_s *b)
{
    if (b->exec) cudaGraphExecDestroy(b->exec);
    if (b->graph) cudaGraphDestroy(b->graph);
    if (b->cap) cudaStreamDestroy(b->cap);
    if (b->side) cudaStreamDestroy(b->side);
    if (b->fork) cudaEventDestroy(b->fork);
    if (b->join) cudaEventDestroy(b->join);
    cudaFree(b->planes);
    cudaFree(b->d_maps);
    cudaFree(b->d_jobs);
    cudaFree(b->d_items);
    cudaFree(b->d_cta_begin);
    cudaFree(b->d_dec);
    cudaFree(b->d_dmaps);
    cudaFree(b->d_djobs);
    cudaFree(b->partials);
    cudaFree(b->sums);
    cudaFree(b->d_sjobs);
    small_scratch_free(&b->small);
    cudaFree(b->d_pjobs);
    cudaFree(b->d_pmaps);
    cudaFree(b->d_err);
    if (b->h_err) cudaFreeHost(b->h_err);
    cudaGetLastError();
    delete b;
}

// Enqueue one run: clear split outputs, decode all jobs, correlate all items.
cudaError_t enqueue_run(xeng_batch_s *b, cudaStream_t s)
{
    // The single-pass jobs of one kernel, in job order, on stream st.
    cudaError_t e = cudaSuccess;
    auto run_single = [&](bool small, cudaStream_t st) {
        for (const auto &jk : b->single) {
            if ((jk.second == kSingleSmall) != small || b->listed[jk.first]) continue;
            const xeng_job_t &jb = b->jobs[jk.first];
            for (int64_t t0 = 0; t0 < jb.n_samples && e == cudaSuccess; t0 += kFusedMaxSamples) {
                const int64_t nt = std::min<int64_t>(kFusedMaxSamples, jb.n_samples - t0);
                e = launch_single_pass(jk.second, jb.block, jb.n_samples, t0, nt, jb.n_freq, jb.n_inputs, 0,
                                       jb.n_freq, jb.out, t0 > 0 ? 1 : 0, &b->small, b->d_err, b->num_sms, st);
            }
        }
    };
    e = cudaMemsetAsync(b->d_err, 0, sizeof(int), s);
    // Two branches: the N <= 256 kernel's jobs (cooperative launches sharing one
    // scratch, so one after another) on a side stream, the rest here; a small
    // job's few CTAs then run beside a large job's tail.
    if (e == cudaSuccess && b->side) {
        e = cudaEventRecord(b->fork, s);
        if (e == cudaSuccess) e = cudaStreamWaitEvent(b->side, b->fork, 0);
        run_single(true, b->side);
        if (e == cudaSuccess) e = cudaEventRecord(b->join, b->side);
    }
    // the longest work first: the pair kernel's persistent launch, whose tail the
    // planes jobs and the side branch fill
    if (e == cudaSuccess && b->n_pjobs > 0)
        e = launch_correlate_pair_listed(b->d_pjobs, b->n_pjobs, b->p_items, b->d_err, b->num_sms, s);
    for (auto &z : b->zero_outs)
        if (e == cudaSuccess) e = cudaMemsetAsync(z.first, 0, z.second, s);
    if (e == cudaSuccess && b->n_djobs > 0)
        e = launch_decode_tma_batch(b->d_dmaps, b->d_djobs, b->n_djobs, b->dtiles, b->d_err, b->num_sms, s);
    if (e == cudaSuccess && b->n_dec > 0) e = launch_decode_batch(b->d_dec, b->n_dec, b->dec_ctas, s);
    if (e == cudaSuccess && b->n_sjobs > 0)
        e = launch_plane_sums_batch(b->d_sjobs, b->n_sjobs, b->sum_entries, b->num_sms, s);
    if (e == cudaSuccess && b->grid > 0) {
        ListArgs L;
        L.maps = b->d_maps;
        L.jobs = b->d_jobs;
        L.items = b->d_items;
        L.cta_begin = b->d_cta_begin;
        L.err = b->d_err;
        L.n_items = b->n_items;
        e = launch_correlate_tc_listed(L, b->grid, s);
    }
    run_single(false, s);
    if (b->side) {
        if (e == cudaSuccess) e = cudaStreamWaitEvent(s, b->join, 0);
    } else {
        run_single(true, s);
    }
    if (e == cudaSuccess) e = cudaMemcpyAsync(b->h_err, b->d_err, sizeof(int), cudaMemcpyDeviceToHost, s);
    return e;
}

// A channel's upper-triangle tile pairs (I <= J) in the requested order.
std::vector<std::pair<int, int>> tile_order(int nt, int order)
{
    std::vector<std::pair<int, int>> v;
    for (int I = 0; I < nt; I++)
        for (int J = I; J < nt; J++) v.push_back({I, J});
    auto morton = [](int I, int J) {
        uint32_t z = 0;
        for (int k = 0; k < 16; k++) z |= (uint32_t)((I >> k) & 1) << (2 * k + 1) | (uint32_t)((J >> k) & 1) << (2 * k);
        return z;
    };
    if (order == XENG_TILES_DIAGONAL)
        std::stable_sort(v.begin(), v.end(), [](const std::pair<int, int> &x, const std::pair<int, int> &y) {
            return x.second - x.first < y.second - y.first;
        });
    else if (order == XENG_TILES_MORTON)
        std::stable_sort(v.begin(), v.end(), [&](const std::pair<int, int> &x, const std::pair<int, int> &y) {
            return morton(x.first, x.second) < morton(y.first, y.second);
        });
    return v;
}

int plan(xeng_batch_s *b)
{
    const int n = (int)b->jobs.size();
    std::vector<int64_t> off(n), n_pad(n), t_pad(n), poff(n, -1), soff(n, -1);
    std::vector<char> single(n, 0);
    const int force = single_pass_force_from_env();
    b->listed.assign(n, 0);
    std::vector<int> pj;  // the pair kernel's listed jobs
    for (int j = 0; j < n; j++) {
        const int k = single_pass_kernel(b->jobs[j].block, b->jobs[j].n_inputs, force, true);
        if (k) {
            single[j] = 1;
            b->single.push_back({j, k});
            if (k == kSinglePair && b->jobs[j].n_samples <= kFusedMaxSamples) {
                b->listed[j] = 1;
                pj.push_back(j);
            }
        }
    }
    if (!pj.empty()) {
        // longest jobs (most stages) first; each job's items after the previous job's
        std::stable_sort(pj.begin(), pj.end(), [&](int x, int y) { return b->jobs[x].n_samples > b->jobs[y].n_samples; });
        std::vector<CUtensorMap> pmaps(pj.size());
        std::vector<PairJob> pjobs(pj.size());
        const int stage = single_pass_stage(kSinglePair);
        int64_t item0 = 0;
        for (size_t k = 0; k < pj.size(); k++) {
            const xeng_job_t &jb = b->jobs[pj[k]];
            if (encode_pair_map(&pmaps[k], jb.block, jb.n_samples, jb.n_freq, jb.n_inputs) != cudaSuccess)
                return XENG_ERR_CUDA;
            const int32_t nt2 = (jb.n_inputs + 255) / 256;
            PairJob &p = pjobs[k];
            p.map = nullptr;  // set once the maps are in device memory
            p.acc = jb.out;
            p.N = jb.n_inputs;
            p.nt = (int32_t)jb.n_samples;
            p.n_k = (int32_t)((jb.n_samples + stage - 1) / stage);
            p.nt2 = nt2;
            p.pairs_per_ch = nt2 * (nt2 + 1) / 2;
            p.item0 = (int32_t)item0;
            item0 += (int64_t)jb.n_freq * p.pairs_per_ch;
            if (item0 > 2147483647LL) return XENG_ERR_RANGE;
        }
        cudaError_t e0 = upload(&b->d_pmaps, pmaps);
        for (size_t k = 0; k < pj.size(); k++) pjobs[k].map = b->d_pmaps + k;
        if (e0 == cudaSuccess) e0 = upload(&b->d_pjobs, pjobs);
        if (e0 != cudaSuccess) return status_of(e0);
        b->n_pjobs = (int)pj.size();
        b->p_items = item0;
    }
    int64_t total = 0, ptotal = 0, stotal = 0;
    for (int j = 0; j < n; j++) {
        if (single[j]) continue;
        const xeng_job_t &jb = b->jobs[j];
        n_pad[j] = round_up(jb.n_inputs, kTile);
        t_pad[j] = round_up(jb.n_samples, kTile);
        off[j] = total;
        total += round_up((int64_t)jb.n_freq * 2 * n_pad[j] * t_pad[j], 1024);
        if (decode_tma_ok(jb.block, jb.n_inputs)) {  // raw-nibble planes: room for the nibble sums
            poff[j] = ptotal;
            soff[j] = stotal;
            ptotal += (int64_t)jb.n_freq * (t_pad[j] / kTile) * n_pad[j];
            stotal += (int64_t)jb.n_freq * n_pad[j];
        }
    }
    b->planes_bytes = total;
    cudaError_t e = cudaMalloc(&b->planes, (size_t)std::max<int64_t>(total, 1));
    if (e == cudaSuccess && ptotal > 0) e = cudaMalloc(&b->partials, (size_t)ptotal * sizeof(int2));
    if (e == cudaSuccess && stotal > 0) e = cudaMalloc(&b->sums, (size_t)stotal * sizeof(int2));
    if (e != cudaSuccess) return status_of(e);
    std::vector<SumJob> sjobs;

    std::vector<CUtensorMap> maps(n);
    std::vector<JobDesc> jd(n);
    std::vector<DecodeJob> dj;
    std::vector<CUtensorMap> dmaps;
    std::vector<DecTmaJob> djobs;
    int64_t dtiles = 0;
    const int maxc = b->opts.max_chunks_per_item;
    struct Cand { WorkItem w; double cost; int64_t order; };
    std::vector<Cand> cand;
    int64_t cta0 = 0;
    for (int j = 0; j < n; j++) {
        if (single[j]) continue;
        const xeng_job_t &jb = b->jobs[j];
        uint8_t *pl = b->planes + off[j];
        e = encode_planes_map(&maps[j], pl, t_pad[j], (int64_t)jb.n_freq * 2 * n_pad[j]);
        if (e != cudaSuccess) return status_of(e);
        const int n_k = (int)(t_pad[j] / kTile);
        CUtensorMap rmap, pmap;
        const bool tma = encode_decode_tma_maps(jb.block, jb.n_samples, jb.n_freq, jb.n_inputs, pl, t_pad[j],
                                                n_pad[j], &rmap, &pmap);
        const bool raw = tma && poff[j] >= 0;
        // raw-nibble items span at most kFusedMaxSamples samples (exact f32 sums)
        const int maxc_j = raw ? std::min(maxc, kFusedMaxSamples / kTile) : maxc;
        const int ns = (n_k + maxc_j - 1) / maxc_j;
        jd[j].out = jb.out;
        jd[j].n_pad = (int32_t)n_pad[j];
        jd[j].N = jb.n_inputs;
        jd[j].mode = ns > 1 ? 2 : 0;  // split tiles add atomically into zeroed outputs
        jd[j].n_samples = (int32_t)jb.n_samples;
        jd[j].sums = raw ? b->sums + soff[j] : nullptr;
        if (raw) {
            SumJob sj;
            sj.partials = b->partials + poff[j];
            sj.sums = b->sums + soff[j];
            sj.first = b->sum_entries;
            sj.n_tb = n_k;
            sj.part_n_tb = n_k;
            sj.n_pad = (int32_t)n_pad[j];
            sj.pad_ = 0;
            sjobs.push_back(sj);
            b->sum_entries += (int64_t)jb.n_freq * n_pad[j];
        }
        if (tma) {
            DecTmaJob dt;
            dt.tile0 = dtiles;
            dt.T = jb.n_samples;
            dt.n_ib = (int32_t)(n_pad[j] / kTile);
            dt.n_tb = (int32_t)(t_pad[j] / kTile);
            dt.F = jb.n_freq;
            dt.N = jb.n_inputs;
            dt.n_pad = (int32_t)n_pad[j];
            dt.x0 = 0;
            dt.partials = raw ? b->partials + poff[j] : nullptr;
            dt.part_n_tb = dt.n_tb;
            dt.pad_ = 0;
            dtiles += (int64_t)dt.n_ib * dt.F * dt.n_tb;
            djobs.push_back(dt);
            dmaps.push_back(rmap);
            dmaps.push_back(pmap);
        } else {
            DecodeJob d;
            d.block = jb.block;
            d.planes = pl;
            d.T = jb.n_samples;
            d.t_pad = t_pad[j];
            d.pitch = t_pad[j];
            d.n_pad = n_pad[j];
            d.cta0 = cta0;
            d.F = jb.n_freq;
            d.N = jb.n_inputs;
            d.vec_ok = decode_vec_ok(jb.block, jb.n_inputs);
            d.pad_ = 0;
            dj.push_back(d);
            cta0 += decode_ctas(t_pad[j], n_pad[j], jb.n_freq);
        }
        if (ns > 1) b->zero_outs.push_back({jb.out, (size_t)jb.n_freq * n_baselines(jb.n_inputs) * 8});
        const int nt = (int)(n_pad[j] / kTile);
        const std::vector<std::pair<int, int>> order = tile_order(nt, b->opts.tile_order);
        for (int f = 0; f < jb.n_freq; f++)
            for (const auto &IJ : order)
                for (int sp = 0; sp < ns; sp++) {
                    const int I = IJ.first, J = IJ.second;
                    Cand c;
                    c.w.job = j;
                    c.w.fl = f;
                    c.w.I = (int16_t)I;
                    c.w.J = (int16_t)J;
                    c.w.kc0 = sp * maxc_j;
                    c.w.kc1 = std::min(n_k, (sp + 1) * maxc_j);
                    // MMA time per chunk, plus a fixed cost for the epilogue and pipeline fill
                    c.cost = (double)(c.w.kc1 - c.w.kc0) + 2.0;
                    c.order = (int64_t)cand.size();
                    cand.push_back(c);
                }
    }
    b->dec_ctas = cta0;
    b->n_sjobs = (int)sjobs.size();
    b->n_dec = (int)dj.size();
    b->n_djobs = (int)djobs.size();
    b->dtiles = dtiles;
    b->n_items = (int64_t)cand.size();
    if (cand.size() > 2147483647ull) return XENG_ERR_RANGE;

    // assignment to persistent CTAs
    const int P = (int)std::max<int64_t>(1, std::min<int64_t>(b->num_sms, (int64_t)cand.size()));
    std::vector<std::vector<int64_t>> per(P);
    std::vector<double> load(P, 0.0);
    typedef std::pair<double, int> LoadCta;
    if (b->opts.policy == XENG_SCHED_ROUND_ROBIN) {
        for (size_t k = 0; k < cand.size(); k++) {
            per[k % P].push_back((int64_t)k);
            load[k % P] += cand[k].cost;
        }
    } else if (b->opts.policy == XENG_SCHED_ORDERED) {
        // items in job / channel / tile order, each to the CTA expected to be
        // free first: the CTAs advance through the list together, as with a
        // shared work queue, so at any time they work on neighbouring tiles of
        // the same channel and share its operands in L2
        std::priority_queue<LoadCta, std::vector<LoadCta>, std::greater<LoadCta>> heap;
        for (int c = 0; c < P; c++) heap.push({0.0, c});
        for (size_t k = 0; k < cand.size(); k++) {
            LoadCta t = heap.top();
            heap.pop();
            per[t.second].push_back((int64_t)k);
            t.first += cand[k].cost;
            load[t.second] = t.first;
            heap.push(t);
        }
    } else {
        std::vector<int64_t> idx(cand.size());
        for (size_t k = 0; k < idx.size(); k++) idx[k] = (int64_t)k;
        std::stable_sort(idx.begin(), idx.end(), [&](int64_t x, int64_t y) { return cand[x].cost > cand[y].cost; });
        std::priority_queue<LoadCta, std::vector<LoadCta>, std::greater<LoadCta>> heap;
        for (int c = 0; c < P; c++) heap.push({0.0, c});
        for (int64_t k : idx) {
            LoadCta t = heap.top();
            heap.pop();
            per[t.second].push_back(k);
            t.first += cand[k].cost;
            load[t.second] = t.first;
            heap.push(t);
        }
        for (auto &v : per) std::sort(v.begin(), v.end());  // job / channel / tile order within a CTA
    }
    std::vector<WorkItem> items;
    items.reserve(cand.size());
    std::vector<int32_t> begin(P + 1, 0);
    double sum = 0, mx = 0;
    for (int c = 0; c < P; c++) {
        begin[c] = (int32_t)items.size();
        for (int64_t k : per[c]) items.push_back(cand[k].w);
        sum += load[c];
        mx = std::max(mx, load[c]);
    }
    begin[P] = (int32_t)items.size();
    b->grid = cand.empty() ? 0 : P;
    b->max_load = mx;
    b->mean_load = P ? sum / P : 0;

    e = upload(&b->d_maps, maps);
    if (e == cudaSuccess) e = upload(&b->d_jobs, jd);
    if (e == cudaSuccess) e = upload(&b->d_items, items);
    if (e == cudaSuccess) e = upload(&b->d_cta_begin, begin);
    if (e == cudaSuccess) e = upload(&b->d_dec, dj);
    if (e == cudaSuccess) e = upload(&b->d_dmaps, dmaps);
    if (e == cudaSuccess) e = upload(&b->d_djobs, djobs);
    if (e == cudaSuccess) e = upload(&b->d_sjobs, sjobs);
    return status_of(e);
}

uint64_t batch_signature(const xeng_job_t *jobs, int n, int num_sms)
{
    uint64_t h = 1469598103934665603ull;  // FNV-1a over the jobs' shapes
    auto mix = [&](uint64_t v) {
        for (int k = 0; k < 8; k++) {
            h ^= (v >> (8 * k)) & 0xFF;
            h *= 1099511628211ull;
        }
    };
    mix((uint64_t)num_sms);
    for (int j = 0; j < n; j++) {
        mix((uint64_t)jobs[j].n_inputs);
        mix((uint64_t)jobs[j].n_freq);
        mix((uint64_t)jobs[j].n_samples);
    }
    return h;
}

}  // namespace

extern "C" {

int xeng_batch_create(const xeng_job_t *jobs, int32_t n_jobs, const xeng_batch_opts_t *opts, xeng_batch_t *out)
{
    if (!out || !jobs || n_jobs < 1) return XENG_ERR_ARG;
    int dev = 0, major = 0, minor = 0, sms = 0;
    if (cudaGetDevice(&dev) != cudaSuccess ||
        cudaDeviceGetAttribute(&major, cudaDevAttrComputeCapabilityMajor, dev) != cudaSuccess ||
        cudaDeviceGetAttribute(&minor, cudaDevAttrComputeCapabilityMinor, dev) != cudaSuccess ||
        cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess) {
        cudaGetLastError();
        return XENG_ERR_UNSUPPORTED;
    }
    if (major != 10 || minor != 3) return XENG_ERR_UNSUPPORTED;
    xeng_batch_opts_t o;
    o.max_chunks_per_item = kMaxChunkSamples / kTile;
    o.policy = XENG_SCHED_LPT;
    o.use_graph = 1;
    o.tile_order = XENG_TILES_ROW_MAJOR;
    if (opts) {
        o = *opts;
        if (o.max_chunks_per_item <= 0 || o.max_chunks_per_item > kMaxChunkSamples / kTile)
            o.max_chunks_per_item = kMaxChunkSamples / kTile;
        if (o.policy != XENG_SCHED_LPT && o.policy != XENG_SCHED_ROUND_ROBIN && o.policy != XENG_SCHED_ORDERED)
            return XENG_ERR_ARG;
        if (o.tile_order != XENG_TILES_ROW_MAJOR && o.tile_order != XENG_TILES_DIAGONAL &&
            o.tile_order != XENG_TILES_MORTON)
            return XENG_ERR_ARG;
    }
    for (int j = 0; j < n_jobs; j++) {
        const xeng_job_t &jb = jobs[j];
        if (!jb.block || !jb.out || (reinterpret_cast<uintptr_t>(jb.out) & 7) != 0) return XENG_ERR_ARG;
        if (jb.n_inputs < 1 || jb.n_inputs > XENG_MAX_INPUTS || jb.n_freq < 1 || jb.n_samples < 1 ||
            jb.n_samples > XENG_MAX_T_INTEG)
            return XENG_ERR_RANGE;
        if (!on_device(jb.block) || !on_device(jb.out)) return XENG_ERR_ARG;
    }
    xeng_batch_s *b = new (std::nothrow) xeng_batch_s;
    if (!b) return XENG_ERR_NOMEM;
    b->jobs.assign(jobs, jobs + n_jobs);
    b->opts = o;
    b->device = dev;
    b->num_sms = sms;
    int st = plan(b);
    cudaError_t e = cudaSuccess;
    if (st == XENG_OK) e = cudaMalloc(&b->d_err, sizeof(int));
    if (st == XENG_OK && e == cudaSuccess) e = cudaMallocHost(&b->h_err, sizeof(int));
    if (st == XENG_OK && e == cudaSuccess) e = prepare_correlate_tc_listed();
    if (st == XENG_OK && e == cudaSuccess) e = prepare_decode_tma_batch();
    if (st == XENG_OK && e == cudaSuccess) e = cudaStreamCreateWithFlags(&b->cap, cudaStreamNonBlocking);
    bool small = false, other = false;
    for (const auto &jk : b->single) (jk.second == kSingleSmall ? small : other) = true;
    if (st == XENG_OK && e == cudaSuccess && small) {  // allocated (flags zeroed) before any capture
        e = small_scratch_alloc(&b->small, b->num_sms, b->cap);
        if (e == cudaSuccess) e = cudaStreamSynchronize(b->cap);
    }
    if (st == XENG_OK && e == cudaSuccess && small && (other || b->grid > 0)) {
        e = cudaStreamCreateWithFlags(&b->side, cudaStreamNonBlocking);
        if (e == cudaSuccess) e = cudaEventCreateWithFlags(&b->fork, cudaEventDisableTiming);
        if (e == cudaSuccess) e = cudaEventCreateWithFlags(&b->join, cudaEventDisableTiming);
    }
    if (st == XENG_OK && e == cudaSuccess && o.use_graph) {
        e = cudaStreamBeginCapture(b->cap, cudaStreamCaptureModeThreadLocal);
        if (e == cudaSuccess) {
            cudaError_t er = enqueue_run(b, b->cap);
            e = cudaStreamEndCapture(b->cap, &b->graph);
            if (e == cudaSuccess) e = er;
        }
        if (e == cudaSuccess) e = cudaGraphInstantiate(&b->exec, b->graph, 0);
    }
    if (st == XENG_OK && e != cudaSuccess) st = status_of(e);
    if (st != XENG_OK) {
        free_batch(b);
        return st;
    }
    *b->h_err = 0;
    *out = b;
    return XENG_OK;
}

int xeng_batch_run(xeng_batch_t b, void *stream)
{
    if (!b) return XENG_ERR_ARG;
    if (b->sticky != XENG_OK) return b->sticky;
    if (*(volatile int *)b->h_err != 0) return (b->sticky = XENG_ERR_TIMEOUT);
    cudaStream_t s = (cudaStream_t)stream;
    cudaError_t e = b->exec ? cudaGraphLaunch(b->exec, s) : enqueue_run(b, s);
    if (e != cudaSuccess) return (b->sticky = status_of(e));
    return XENG_OK;
}

int xeng_batch_info(xeng_batch_t b, xeng_batch_info_t *info)
{
    if (!b || !info) return XENG_ERR_ARG;
    info->n_jobs = (int32_t)b->jobs.size();
    info->n_items = b->n_items;
    info->grid = b->grid;
    info->decode_ctas = b->dec_ctas + b->dtiles;
    info->planes_bytes = b->planes_bytes;
    info->max_chunks_per_item = b->opts.max_chunks_per_item;
    info->policy = b->opts.policy;
    info->tile_order = b->opts.tile_order;
    info->load_imbalance = b->mean_load > 0 ? b->max_load / b->mean_load : 1.0;
    return XENG_OK;
}

void xeng_batch_destroy(xeng_batch_t b)
{
    if (!b) return;
    cudaDeviceSynchronize();
    free_batch(b);
}

int xeng_batch_autotune(const xeng_job_t *jobs, int32_t n_jobs, const char *cache_path, int32_t reps,
                        xeng_batch_opts_t *best, double *best_ms)
{
    if (!jobs || n_jobs < 1 || !best) return XENG_ERR_ARG;
    int dev = 0, sms = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess) {
        cudaGetLastError();
        return XENG_ERR_UNSUPPORTED;
    }
    const uint64_t sig = batch_signature(jobs, n_jobs, sms);
    if (cache_path) {
        FILE *fp = fopen(cache_path, "r");
        if (fp) {
            char line[256];
            while (fgets(line, sizeof(line), fp)) {
                unsigned long long s = 0;
                int mc = 0, pol = 0, ord = 0;
                double ms = 0;
                if (sscanf(line, "{\"sig\": \"%llx\", \"max_chunks\": %d, \"policy\": %d, \"tile_order\": %d, \"ms\": %lf}",
                           &s, &mc, &pol, &ord, &ms) == 5 &&
                    (uint64_t)s == sig) {
                    best->max_chunks_per_item = mc;
                    best->policy = pol;
                    best->use_graph = 1;
                    best->tile_order = ord;
                    if (best_ms) *best_ms = ms;
                    fclose(fp);
                    return 1;  // from the cache
                }
            }
            fclose(fp);
        }
    }
    if (reps < 1) reps = 3;
    const int chunks[] = {16, 32, 64, 128, 256, 512};
    const int policies[] = {XENG_SCHED_LPT, XENG_SCHED_ROUND_ROBIN, XENG_SCHED_ORDERED};
    cudaStream_t s;
    if (cudaStreamCreateWithFlags(&s, cudaStreamNonBlocking) != cudaSuccess) return XENG_ERR_CUDA;
    cudaEvent_t e0, e1;
    cudaEventCreate(&e0);
    cudaEventCreate(&e1);
    // Every candidate is timed in two passes, forward and then in reverse
    // order, and keeps its better time: the GPU warms up and meets its power
    // cap during tuning, which would otherwise favour the candidates timed
    // first.
    std::vector<xeng_batch_opts_t> cands;
    for (int pol : policies)
        for (int mc : chunks) {
            xeng_batch_opts_t o;
            o.max_chunks_per_item = mc;
            o.policy = pol;
            o.use_graph = 1;
            o.tile_order = XENG_TILES_ROW_MAJOR;
            cands.push_back(o);
        }
    // time cands[from, to) in two passes; each keeps its better time (< 0: failed)
    std::vector<double> t_best(cands.size(), -1.0);
    auto time_range = [&](size_t from, size_t to) {
        for (int pass = 0; pass < 2; pass++)
            for (size_t c = from; c < to; c++) {
                const size_t k = pass == 0 ? c : to - 1 - (c - from);
                xeng_batch_t b = nullptr;
                if (xeng_batch_create(jobs, n_jobs, &cands[k], &b) != XENG_OK) continue;
                int st = xeng_batch_run(b, s);
                cudaEventRecord(e0, s);
                for (int r = 0; r < reps && st == XENG_OK; r++) st = xeng_batch_run(b, s);
                cudaEventRecord(e1, s);
                float ms = 0;
                if (st == XENG_OK && cudaEventSynchronize(e1) == cudaSuccess &&
                    cudaEventElapsedTime(&ms, e0, e1) == cudaSuccess && *(volatile int *)b->h_err == 0) {
                    const double t = ms / reps;
                    if (t_best[k] < 0 || t < t_best[k]) t_best[k] = t;
                }
                xeng_batch_destroy(b);
            }
    };
    auto pick = [&](double &best_t) {
        int at = -1;
        for (size_t k = 0; k < cands.size(); k++)
            if (t_best[k] >= 0 && (at < 0 || t_best[k] < best_t)) {
                best_t = t_best[k];
                at = (int)k;
            }
        return at;
    };
    time_range(0, cands.size());
    double best_t = -1;
    int at = pick(best_t);
    if (at >= 0) {
        // the winner's schedule with the other tile orders
        const size_t n0 = cands.size();
        for (int ord : {XENG_TILES_DIAGONAL, XENG_TILES_MORTON}) {
            xeng_batch_opts_t o = cands[at];
            o.tile_order = ord;
            cands.push_back(o);
            t_best.push_back(-1.0);
        }
        time_range(n0, cands.size());
        at = pick(best_t);
    }
    int st_all = XENG_ERR_CUDA;
    if (at >= 0) {
        *best = cands[at];
        st_all = XENG_OK;
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    cudaStreamDestroy(s);
    if (st_all != XENG_OK) return st_all;
    if (best_ms) *best_ms = best_t;
    if (cache_path) {
        FILE *fp = fopen(cache_path, "a");
        if (fp) {
            fprintf(fp, "{\"sig\": \"%016llx\", \"max_chunks\": %d, \"policy\": %d, \"tile_order\": %d, \"ms\": %.6f}\n",
                    (unsigned long long)sig, best->max_chunks_per_item, best->policy, best->tile_order, best_t);
            fclose(fp);
        }
    }
    return XENG_OK;
}

}  // extern "C"
