// lbm_noalloc.cu -- observables of a caller-held state without allocating any memory.
//
// Some callers cannot let a library allocate device memory while they run: code that is
// being recorded into a CUDA graph (cudaMalloc may not be called during stream capture),
// real-time loops that must not take the allocator's locks or risk its latency, and host
// applications that reserve the whole device up front through their own pool, where an
// allocation from elsewhere fails or fragments that pool.  For them lbm_observables_noalloc
// computes the same observables as lbm_observables, but every scratch buffer it needs lives
// in one file-scope device array of fixed size, LBM_NOALLOC_SCRATCH_BYTES, which each GPU
// that loads the library holds until the process exits.  The caller passes the populations
// and the output buffer.
#include <atomic>

#include "lbm.h"
#include "lbm_consts.h"
#include "lbm_internal.h"

using namespace lbm;

namespace {

// The scratch array.  Host code must not use its name as a device address (on the host it
// names a stand-in object); the device address comes from cudaGetSymbolAddress below.
static __device__ __align__(256) unsigned char g_scratch[LBM_NOALLOC_SCRATCH_BYTES];

constexpr int MAX_DEVICES = 64;
// device address of g_scratch per device, as last looked up (kept for calls made during a
// stream capture, when no lookup is made)
std::atomic<void*> g_scratch_ptr[MAX_DEVICES];

size_t align256(size_t n) { return (n + 255) / 256 * 256; }

}  // namespace

extern "C" int lbm_observables_noalloc(const double* f, int nx, int nz, int n_species, int z_boundary,
                                       const lbm_params* p, double* out, void* stream) {
    if (!f || !out || !p) return LBM_EINVAL;
    if (nx < 1 || nz < 1 || nx > 65536 || nz > 65536 || (n_species != 1 && n_species != 2) ||
        (z_boundary != LBM_PERIODIC && z_boundary != LBM_BOUNCEBACK))
        return LBM_EINVAL;
    if (lbm_validate_params(p, n_species) != LBM_OK) return LBM_EINVAL;
    // scratch layout: row partials, column partials, scalar slots, wall sums, ticket, flag
    const int nxpart = (nx + TPX - 1) / TPX, nzpart = (nz + TPZ - 1) / TPZ;
    const size_t b_row = align256((size_t)nz * nxpart * NQR * sizeof(double));
    const size_t b_col = align256((size_t)nx * nzpart * NQC * sizeof(double));
    const size_t b_slots = align256((size_t)(nx + nz) * 5 * sizeof(double));
    const size_t b_small = 256;  // wall sums (2 doubles), ticket, flag
    const size_t need = b_row + b_col + b_slots + b_small;
    if (need > (size_t)LBM_NOALLOC_SCRATCH_BYTES) return LBM_ENOMEM;  // does not fit the fixed scratch

    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= MAX_DEVICES) return LBM_ECUDA;
    const cudaStream_t st = static_cast<cudaStream_t>(stream);
    // The array's device address, looked up with this device current.  It is looked up again on
    // every call made outside a stream capture, so a device reset (which reloads the module at
    // another address) is followed; during a capture the address of the last lookup is used.
    cudaStreamCaptureStatus cap = cudaStreamCaptureStatusNone;
    if (cudaStreamIsCapturing(st, &cap) != cudaSuccess) return LBM_ECUDA;
    void* ptr = g_scratch_ptr[dev].load();
    if (cap == cudaStreamCaptureStatusNone || !ptr) {
        ptr = nullptr;
        if (cudaGetSymbolAddress(&ptr, g_scratch) != cudaSuccess || !ptr) return LBM_ECUDA;
        g_scratch_ptr[dev].store(ptr);
    }
    unsigned char* base = static_cast<unsigned char*>(ptr);
    ObsPtrs O;
    O.part_row = base;
    O.part_col = base + b_row;
    double* slots = reinterpret_cast<double*>(base + b_row + b_col);
    double* walls = reinterpret_cast<double*>(base + b_row + b_col + b_slots);
    unsigned* ticket = reinterpret_cast<unsigned*>(walls + 2);
    O.flag = reinterpret_cast<int*>(ticket + 1);
    O.fields = nullptr;

    StepConst<double> C;
    const double rr[2] = {0.0, 0.0};  // plain FP64 populations
    fill_step_const<double>(C, *p, nx, nz, nx, (long long)nx * nz, n_species, z_boundary, rr);
    // the array keeps the previous call's contents: the ticket and the flag must start at zero
    cudaError_t e = cudaMemsetAsync(walls, 0, b_small, st);
    if (e == cudaSuccess) e = launch_tile<double>(n_species, M_OBS, TPZ, f, nullptr, C, O, st);
    if (e == cudaSuccess)
        e = launch_reduce((int)sizeof(double), O, nxpart, nzpart, nx, nz, z_boundary, ticket, out, nullptr, slots,
                          nullptr, 0, true, nullptr, 0, st);
    return e == cudaSuccess ? LBM_OK : LBM_ECUDA;
}
