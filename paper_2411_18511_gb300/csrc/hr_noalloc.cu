// hr_noalloc.cu -- |v|^2 of a packed FP64 spinor field without any allocation.
//
// Every other entry point of this library needs an hr_ctx, and creating one
// calls cudaMalloc for the context's reduction scratch.  Some callers cannot do
// that: code running where the CUDA allocator is off limits (a host that
// pre-reserves all device memory for its own pool and forbids further device
// allocations, plug-ins that may not touch the process's allocator, or code
// paths that must not allocate between their set-up and tear-down).  This file
// gives them one reduction that needs neither a context nor a workspace: its
// block partial sums and its completion counter live in a fixed device array
// declared at file scope, which every GPU that loads the library holds until
// the process exits.
#include <atomic>

#include "hr_host.h"

using namespace hr;

namespace {

// Scratch: kNoAllocBlocks partial sums per right-hand side, plus a counter.
constexpr int kNoAllocBlocks = 1024;
constexpr int kNoAllocDoubles = kNoAllocBlocks * kMaxRhs; // 32768 doubles = 256 KiB
struct NoAllocScratch {
    double partials[kNoAllocDoubles];
    unsigned counter;
};
static __device__ __align__(256) NoAllocScratch g_noalloc_scratch;

// Device address of the scratch, looked up once per device (host code may
// not pass the symbol itself: in host code its name is only a stand-in).
// Atomic entries: two host threads making their first call at the same time
// both look the address up and store the same value.  A cudaDeviceReset on
// the device invalidates the entry; a failed launch clears it, so the next
// call looks the address up again.
constexpr int kMaxDevices = 64;
static std::atomic<NoAllocScratch *> g_scratch_addr[kMaxDevices];

template <int NC>
__global__ void __launch_bounds__(256) k_norm2_noalloc(Geom g, const void *v, NoAllocScratch *scr, double *result)
{
    using T = PrecTraits<kF64>::T;
    const int nv = g.vh << g.lrhs;
    SqAcc<T> acc;
    for (int j = blockIdx.x * blockDim.x + threadIdx.x; j < nv; j += gridDim.x * blockDim.x) {
        cpx<T> a[4][NC];
        load_spinor<NC, kF64>(v, g.nblk_s, j, a);
#pragma unroll
        for (int s = 0; s < 4; ++s)
#pragma unroll
            for (int c = 0; c < NC; ++c) {
                acc.add(a[s][c].re);
                acc.add(a[s][c].im);
            }
    }
    __shared__ double smem[32 * 32];
    __shared__ double sums[32];
    RedSlot slot;
    slot.partials = scr->partials;
    slot.counter = &scr->counter;
    slot.group_counters = nullptr; // one level: the fixed scratch has no group slots
    slot.group_partials = nullptr;
    if (grid_reduce(acc, g.nrhs, slot, sums, smem)) {
        if (threadIdx.x < g.nrhs) result[threadIdx.x] = sums[threadIdx.x];
    }
}

} // namespace

extern "C" hr_status hr_norm2_noalloc(hr_lattice lat, hr_rep rep, int n_rhs, const void *v, double *result,
                                      hr_stream stream)
{
    if (!valid_rep(rep)) return HR_ERR_INVALID_ARG;
    if (!v || !result || ((uintptr_t)v & 15u)) return HR_ERR_INVALID_ARG; // packed: 16-byte vectors
    // the fixed scratch holds kMaxRhs partial sums per block: more RHS do not fit
    if (n_rhs > kMaxRhs) return HR_ERR_WORKSPACE;
    if (n_rhs < 1 || (n_rhs & (n_rhs - 1))) return HR_ERR_UNSUPPORTED;
    // the same codes as the context-based calls (a null ctx records no message)
    if (hr_status st = validate_lattice(nullptr, lat, n_rhs)) return st;
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= kMaxDevices) {
        cudaGetLastError();
        return HR_ERR_CUDA;
    }
    cudaStream_t s = (cudaStream_t)stream;
    // the kernel runs on the current device, whose scratch it is given: a
    // stream of another device is an argument error
    if (s) {
        int sdev = -1;
        if (cudaStreamGetDevice(s, &sdev) != cudaSuccess) {
            cudaGetLastError();
            return HR_ERR_INVALID_ARG;
        }
        if (sdev != dev) return HR_ERR_INVALID_ARG;
    }
    // set-up, once per device: the first call on a device must not be inside a
    // stream capture (it queries the symbol address, which under lazy module
    // loading also loads this file's module and places the array)
    NoAllocScratch *scr = g_scratch_addr[dev].load();
    if (!scr) {
        void *ptr = nullptr;
        cudaError_t e = cudaGetSymbolAddress(&ptr, g_noalloc_scratch);
        if (e != cudaSuccess || !ptr) {
            cudaGetLastError();
            return HR_ERR_CUDA;
        }
        scr = (NoAllocScratch *)ptr;
        g_scratch_addr[dev].store(scr);
    }
    Geom g = make_geom(lat, n_rhs);
    // the grid never exceeds the partial-sum slots of the scratch
    int sms = 0;
    if (cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess) {
        cudaGetLastError();
        return HR_ERR_CUDA;
    }
    int cap = sms > 0 ? sms * 4 : 256;
    if (cap > kNoAllocBlocks) cap = kNoAllocBlocks;
    int grid = grid_for((long long)g.vh << g.lrhs, 256, cap);
    // the scratch keeps the previous call's contents: the counter must start at zero
    if (cudaMemsetAsync(&scr->counter, 0, sizeof(unsigned), s) != cudaSuccess) {
        cudaGetLastError();
        return HR_ERR_CUDA;
    }
    if (rep_nc(rep) == 2) k_norm2_noalloc<2><<<grid, 256, 0, s>>>(g, v, scr, result);
    else k_norm2_noalloc<3><<<grid, 256, 0, s>>>(g, v, scr, result);
    if (cudaGetLastError() != cudaSuccess) {
        g_scratch_addr[dev].store(nullptr); // look the address up again next time
        return HR_ERR_CUDA;
    }
    return HR_OK;
}
