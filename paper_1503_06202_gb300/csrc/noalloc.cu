// noalloc.cu -- xeng_correlate_noalloc: the tensor-engine correlation for
// callers that cannot allocate device memory.
//
// Some callers of a correlator cannot call cudaMalloc or cudaFree at the
// point where they correlate: a real-time capture loop whose device memory
// was carved up once at start-up by its own pool (a fresh allocation may fail
// or fragment that pool), or a loop that must not stall, since cudaMalloc and
// cudaFree may synchronize the whole device and break the loop's latency
// budget.  For them this entry point keeps its working memory -- the decoded
// FP8 planes and the kernels' status word -- in one file-scope __device__
// array of fixed size that every GPU loading this library holds until the
// process exits.  The caller passes only the input block and the output.
//
// The array is shared by every call on a device and keeps the last call's
// contents: the decode stage overwrites every byte of the planes a round
// uses, and the status word is zeroed at the start of each call.  Calls that
// overlap on the GPU (two host threads, or two streams) race on the array.
//
// Host code never passes the array's name to a kernel: in host code that
// name is a host-side stand-in, not a device address.  The device address is
// looked up once per device with cudaGetSymbolAddress, with that device
// current, on the first call made on it; make that first call before any
// stream capture.  The address is kept for the life of the process: it does
// not survive cudaDeviceReset, after which this entry point must not be
// called on that device again.
#include <mutex>

#include "../../include/xeng.h"
#include "xeng_internal.h"

namespace {

using namespace xeng;

// The planes take all of XENG_NOALLOC_SCRATCH_BYTES; the status word sits in
// 256 bytes after them (kept apart so the planes stay 256-byte aligned).
constexpr int64_t kPlaneBytes = (int64_t)XENG_NOALLOC_SCRATCH_BYTES;
constexpr int64_t kStatusBytes = 256;
constexpr int kMaxDevices = 64;

static __device__ __align__(256) uint8_t xeng_noalloc_scratch[XENG_NOALLOC_SCRATCH_BYTES + kStatusBytes];

std::mutex g_setup_mutex;
uint8_t *g_scratch_addr[kMaxDevices];  // device address of the array, per device

// Device address of the scratch array on `dev` (which must be current).
int scratch_on(int dev, uint8_t **addr)
{
    if (dev < 0 || dev >= kMaxDevices) return XENG_ERR_UNSUPPORTED;
    std::lock_guard<std::mutex> lock(g_setup_mutex);
    if (!g_scratch_addr[dev]) {
        void *p = nullptr;
        cudaError_t e = cudaGetSymbolAddress(&p, xeng_noalloc_scratch);
        if (e != cudaSuccess || !p) {
            cudaGetLastError();
            return XENG_ERR_CUDA;
        }
        g_scratch_addr[dev] = static_cast<uint8_t *>(p);
    }
    *addr = g_scratch_addr[dev];
    return XENG_OK;
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

}  // namespace

extern "C" int xeng_correlate_noalloc(const uint8_t *block, int64_t n_samples, int32_t n_freq, int32_t n_inputs,
                                      int32_t *out, void *stream)
{
    if (!block || !out || (reinterpret_cast<uintptr_t>(out) & 7) != 0) return XENG_ERR_ARG;
    if (n_inputs < 1 || n_inputs > XENG_MAX_INPUTS || n_freq < 1 || n_samples < 0) return XENG_ERR_RANGE;
    const int64_t n_pad = round_up(n_inputs, kTile);
    const int64_t t_pad = round_up(n_samples > 0 ? n_samples : 1, kTile);
    // one channel's decoded planes over the whole block must fit, and one
    // launch may integrate at most kMaxChunkSamples samples (exact f32 sums)
    if (t_pad > kMaxChunkSamples || 2 * n_pad * t_pad > kPlaneBytes) return XENG_ERR_RANGE;

    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess) {
        cudaGetLastError();
        return XENG_ERR_UNSUPPORTED;
    }
    int major = 0, minor = 0, sms = 0;
    if (cudaDeviceGetAttribute(&major, cudaDevAttrComputeCapabilityMajor, dev) != cudaSuccess ||
        cudaDeviceGetAttribute(&minor, cudaDevAttrComputeCapabilityMinor, dev) != cudaSuccess ||
        cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess) {
        cudaGetLastError();
        return XENG_ERR_UNSUPPORTED;
    }
    if (major != 10 || minor != 3) return XENG_ERR_UNSUPPORTED;
    if (!on_device(block) || !on_device(out)) return XENG_ERR_ARG;

    uint8_t *scratch = nullptr;
    int st = scratch_on(dev, &scratch);
    if (st != XENG_OK) return st;
    uint8_t *planes = scratch;
    int *status = reinterpret_cast<int *>(scratch + kPlaneBytes);

    cudaStream_t s = (cudaStream_t)stream;
    const int64_t N = n_inputs, F = n_freq;
    const int64_t nb2 = N * (N + 1);
    cudaError_t e;
    if (n_samples == 0) {
        e = cudaMemsetAsync(out, 0, (size_t)(F * nb2 * 4), s);
        if (e == cudaSuccess) e = cudaStreamSynchronize(s);
        return e == cudaSuccess ? XENG_OK : XENG_ERR_CUDA;
    }
    e = cudaMemsetAsync(status, 0, sizeof(int), s);
    int64_t group = kPlaneBytes / (2 * n_pad * t_pad);
    if (group > F) group = F;
    if (group > 65535) group = 65535;
    for (int64_t f0 = 0; f0 < F && e == cudaSuccess; f0 += group) {
        const int32_t nf = (int32_t)((F - f0) < group ? (F - f0) : group);
        e = decode_tma_ok(block, (int32_t)N)
                ? launch_decode_tma(block, n_samples, (int32_t)F, (int32_t)N, (int32_t)f0, nf, planes, t_pad, n_pad,
                                    status, sms, s)
                : launch_decode(block, n_samples, (int32_t)F, (int32_t)N, (int32_t)f0, nf, planes, t_pad, n_pad, s);
        if (e != cudaSuccess) break;
        TcArgs a;
        a.planes = planes;
        a.t_pad = t_pad;
        a.n_pad = (int32_t)n_pad;
        a.N = (int32_t)N;
        a.nf = nf;
        a.acc = out + f0 * nb2;
        a.accumulate = 0;
        a.err = status;
        e = launch_correlate_tc(a, sms, s);
    }
    int host_status = 0;
    if (e == cudaSuccess) e = cudaMemcpyAsync(&host_status, status, sizeof(int), cudaMemcpyDeviceToHost, s);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);
    if (e != cudaSuccess) {
        cudaGetLastError();
        return XENG_ERR_CUDA;
    }
    return host_status != 0 ? XENG_ERR_TIMEOUT : XENG_OK;
}
