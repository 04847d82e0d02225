// frost_accel_noalloc: the mixed-precision Newtonian pass of all particles against all
// particles, for callers that cannot allocate device memory.
//
// Some callers cannot call cudaMalloc or any other allocating routine. Examples are code that
// runs under an allocator that forbids new device allocations, code embedded in a larger
// application that owns all device memory, and code that must not allocate in the middle of
// time-critical work. The regular entry points need a frost_ctx, which allocates its state and
// scratch. This entry point instead takes its inputs and output from the caller and keeps
// its scratch in one file-scope device array, g_noalloc_scratch.
//   - Every GPU that loads the library holds this array until the process exits.
//   - The array is shared by every call in the process and keeps the previous call's contents.
//     The only part that must start at zero, the error word, is cleared by each call.
//   - Two calls whose GPU work overlaps (different streams or host threads, no ordering between
//     them) race on the array and give wrong results. Serialise them.
//   - The first call on a device looks up the array's device address (cudaGetSymbolAddress);
//     make that call before any stream capture.  Every call synchronises its stream before it
//     returns, to read the status word of its kernels.
//
// The kernels are the ones the context-based path launches (pack, the FP32 pair kernel with
// float-float separations and compensated sums, the FP64 finalisation); only the scratch and
// the input layout differ.
#include "frost.h"
#include "frost_internal.cuh"

#include <cmath>
#include <cstdarg>
#include <cstdio>
#include <mutex>

using namespace frost;

namespace {

constexpr int kNoallocMaxN = FROST_NOALLOC_MAX_N;
constexpr size_t kRecBytes = (size_t)2 * 16 * kNoallocMaxN;   // two float4 records per particle
constexpr size_t kPartBytes = (size_t)6 * 1024 * 1024;          // split partials (doubles)
constexpr size_t kScratchBytes = kRecBytes + kPartBytes + 256;  // + error word
constexpr int kMaxDevices = 64;

static __device__ __align__(256) unsigned char g_noalloc_scratch[kScratchBytes];

std::mutex g_setup_mutex;
unsigned char *g_scratch_ptr[kMaxDevices] = {nullptr};
int g_num_sm[kMaxDevices] = {0};
// A failure sets the calling thread's message (frost_last_error) in its fixed thread-local
// storage and returns the status; nothing is allocated.
frost_status noalloc_fail(frost_status st, const char *fmt, ...) __attribute__((format(printf, 2, 3)));
frost_status noalloc_fail(frost_status st, const char *fmt, ...)
{
    char buf[kLastErrorBytes];
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(buf, sizeof(buf), fmt, ap);
    va_end(ap);
    set_last_error("frost_accel_noalloc: %s", buf);
    return st;
}

// One-time set-up per device, with that device current: the device address of the scratch
// array (the host-side symbol is only a stand-in) and the SM count.  The address is kept for
// the life of the process; a cudaDeviceReset of that device unloads the library's device code,
// after which the kept address is stale, so the entry point must not be used on that device
// again.
frost_status setup_device(int dev, unsigned char **scratch, int *nsm)
{
    if (dev < 0 || dev >= kMaxDevices) return noalloc_fail(FROST_ECUDA, "device index %d out of range", dev);
    std::lock_guard<std::mutex> lock(g_setup_mutex);
    if (!g_scratch_ptr[dev]) {
        void *p = nullptr;
        const cudaError_t e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
        if (e != cudaSuccess || !p)
            return noalloc_fail(FROST_ECUDA, "cudaGetSymbolAddress failed: %s", cudaGetErrorString(e));
        int n = 0;
        const cudaError_t e2 = cudaDeviceGetAttribute(&n, cudaDevAttrMultiProcessorCount, dev);
        if (e2 != cudaSuccess || n <= 0)
            return noalloc_fail(FROST_ECUDA, "SM count query failed: %s", cudaGetErrorString(e2));
        g_num_sm[dev] = n;
        g_scratch_ptr[dev] = (unsigned char *)p;
    }
    *scratch = g_scratch_ptr[dev];
    *nsm = g_num_sm[dev];
    return FROST_OK;
}

// [n][3] positions and masses -> the float-float records of the mixed Newtonian pass
__global__ void k_pack_noalloc(const double *__restrict__ x, const double *__restrict__ m, int n,
                               float4 *__restrict__ rec, int *__restrict__ err)
{
    const int k = blockIdx.x * blockDim.x + threadIdx.x;
    if (k >= n) return;
    const double px = x[3 * (size_t)k], py = x[3 * (size_t)k + 1], pz = x[3 * (size_t)k + 2];
    const double mk = m[k];
    if (!isfinite(px) || !isfinite(py) || !isfinite(pz) || !(mk > 0.0) || !isfinite(mk))
        atomicOr(err, ERR_NONFINITE);
    const float hx = (float)px, hy = (float)py, hz = (float)pz;
    const float mh = (float)mk;
    rec[k] = make_float4(hx, hy, hz, mh);
    rec[n + k] = make_float4((float)(px - (double)hx), (float)(py - (double)hy),
                             (float)(pz - (double)hz), (float)(mk - (double)mh));
}

}  // namespace

extern "C" frost_status frost_accel_noalloc(int64_t n, const double *m, const double *x, double G,
                                            double eps_soft, double *acc, void *cuda_stream)
{
    clear_last_error();
    if (n < 1 || n > kNoallocMaxN)
        return noalloc_fail(FROST_EINVAL, "n = %lld outside [1, %d] (the size of the static scratch)", (long long)n,
                            kNoallocMaxN);
    if (!m || !x || !acc) return noalloc_fail(FROST_EINVAL, "m, x and acc are required");
    if (!(G > 0.0) || !std::isfinite(G) || !(eps_soft >= 0.0) || !std::isfinite(eps_soft))
        return noalloc_fail(FROST_EINVAL, "G must be finite and positive, eps_soft finite and >= 0");
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return noalloc_fail(FROST_ECUDA, "cudaGetDevice: %s", cudaGetErrorString(e));
    unsigned char *scratch = nullptr;
    int nsm = 0;
    const frost_status st = setup_device(dev, &scratch, &nsm);
    if (st != FROST_OK) return st;

    const cudaStream_t s = (cudaStream_t)cuda_stream;
    float4 *rec = (float4 *)scratch;
    double *part = (double *)(scratch + kRecBytes);
    int *err = (int *)(scratch + kRecBytes + kPartBytes);
    const int ni = (int)n;

    // split the source list only as far as the partial buffer allows
    SplitShape sh = choose_shape(ni, ni, pair_i_per_block(true), pair_blocks_per_sm(PASS_ACC, true), nsm);
    const size_t max_split = kPartBytes / (sizeof(double) * 3 * (size_t)ni);
    if ((size_t)sh.nsplit > max_split) {
        const int tiles = (ni + PAIR_TJ - 1) / PAIR_TJ;
        const int ns = (int)std::max<size_t>(1, max_split);
        sh.j_per_split = ((tiles + ns - 1) / ns) * PAIR_TJ;
        sh.nsplit = (ni + sh.j_per_split - 1) / sh.j_per_split;
    }
    // the partials [nsplit][3][n] and the records [2][n] must fit their parts of the array
    if ((size_t)sh.nsplit * 3 * (size_t)ni * sizeof(double) > kPartBytes || (size_t)2 * ni * sizeof(float4) > kRecBytes)
        return noalloc_fail(FROST_EINVAL, "internal: %d splits of %d particles exceed the static scratch", sh.nsplit, ni);

    e = cudaMemsetAsync(err, 0, sizeof(int), s);
    if (e != cudaSuccess) return noalloc_fail(FROST_ECUDA, "clearing the error word: %s", cudaGetErrorString(e));
    k_pack_noalloc<<<(ni + 255) / 256, 256, 0, s>>>(x, m, ni, rec, err);
    PairArgs a;
    a.irec = rec;
    a.jrec = rec;
    a.n_a = ni;
    a.n_s = ni;
    a.self_pass = 1;
    a.eps2 = eps_soft * eps_soft;
    a.part = part;
    a.shape = sh;
    launch_acc(s, true, a);
    launch_finalize_vec(s, part, sh.nsplit, ni, G, nullptr, acc, err,
                        eps_soft == 0.0 ? ERR_COINCIDENT : ERR_NONFINITE);
    e = cudaGetLastError();
    if (e != cudaSuccess) return noalloc_fail(FROST_ECUDA, "launch: %s", cudaGetErrorString(e));
    int herr = 0;
    e = cudaMemcpyAsync(&herr, err, sizeof(int), cudaMemcpyDeviceToHost, s);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);
    if (e != cudaSuccess) return noalloc_fail(FROST_ECUDA, "reading the error word: %s", cudaGetErrorString(e));
    if (herr & ERR_COINCIDENT) return noalloc_fail(FROST_ECOINCIDENT, "two particles at zero separation");
    if (herr) return noalloc_fail(FROST_ENONFINITE, "non-finite input, non-positive mass or non-finite result");
    return FROST_OK;
}
