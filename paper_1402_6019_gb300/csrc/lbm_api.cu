// lbm_api.cu -- the C ABI of liblbm.so (declared in include/lbm.h).
//
// Owns the device buffers of one simulation, turns lbm_params into the per-step constant
// tables of the kernels, and enqueues the kernels on the context's stream.  Every entry
// point returns a status; nothing throws across the ABI.
#include <stdarg.h>
#include <stddef.h>
#include <stdio.h>
#include <string.h>

#include <algorithm>
#include <array>
#include <atomic>
#include <cmath>
#include <map>
#include <new>
#include <string>
#include <vector>

#include "lbm.h"
#include "lbm_consts.h"
#include "lbm_internal.h"

using namespace lbm;

// The 256-byte tail of a snapshot: the reference densities of the FP32 deviations, the step
// counter, the writer's tag (context serial << 32 | snapshot sequence number) and the shape the
// populations were written for.
struct SnapTail {
    double rho_ref[2];
    long long step;
    unsigned long long tag;
    int nx, nz, ns, precision, n_inst, pad;
};
static_assert(sizeof(SnapTail) <= 256, "snapshot tail");
static std::atomic<unsigned> g_ctx_serial{0};
static const size_t SNAP_CACHE_MAX = 1024;  // remembered snapshot tails per context

struct lbm_ctx {
    lbm_desc d{};
    lbm_params p{};
    int pitch = 0;
    long long plane = 0;
    size_t esize = 0;  // bytes per stored population value
    void* f[2] = {nullptr, nullptr};      // the population buffers (lattice layout origin)
    void* f_raw[2] = {nullptr, nullptr};  // their allocations (f = f_raw + a shift)
    int cur = 0;
    cudaStream_t stream = nullptr;
    bool own_stream = false;
    int nsm = 0;
    SweepGeom geom{};      // fused kernel without observables (M_WRITE, M_FIELDS)
    SweepGeom geom_obs{};  // fused kernel with observables (M_OBS modes)
    GhostGeom ghost{};
    int kernel = LBM_KERNEL_FUSED;  // resolved
    int tile_rows = 8;              // resolved tile height of the FUSED kernel
    int nxpart = 0, nzpart = 0;     // partial-sum groups of the kernel in use
    void* part_row[2] = {nullptr, nullptr};  // partial sums in the populations' precision, one
    void* part_col[2] = {nullptr, nullptr};  // set per population buffer parity
    unsigned* sched = nullptr;  // pull: two pairs of work-item counters, used by alternate launches
    int sched_set = 0;          // the pair the next pull launch uses (the other is zeroed by it)
    // pull: the last observing step's partial sums (in part_*[pending_buf]) still to be reduced;
    // the next pull launch folds the reduction in, a host read flushes it with k_reduce
    bool pending = false;
    bool pending_acc = false;
    int pending_buf = 0;
    unsigned* ticket = nullptr;
    int* flag = nullptr;
    double* out = nullptr;
    double* avg = nullptr;
    double* staging = nullptr;  // (ns + 2) * n doubles
    double* dcheck = nullptr;   // lbm_set_fields: DCHECK_DOUBLES doubles (launch_density_check)
    double* fexport = nullptr;  // ns * 9 * n doubles
    void* adj_scratch = nullptr;  // adjoint: adjoint_scratch_bytes(nx, nz, ns)
    void* adj_lam = nullptr;      // adjoint: second lam buffer, ns * 9 * n doubles
    void* gfield = nullptr;     // two-pass ghost fields
    alignas(64) unsigned char tmap[128] = {};  // two-pass: TMA descriptor of gfield
    bool pull = false;                          // pull layout (LBM_KERNEL_PULL)
    alignas(64) unsigned char pmap_in[2][128] = {};   // pull: load descriptors of f[0], f[1] (tile width 32)
    alignas(64) unsigned char pmap_wide[2][128] = {}; // pull, FP32: the same for tiles of width 64
    int pull_grid[32][2][2] = {};                     // pull: resident CTAs per mode, depth and width (32, 64)
    void* rec = nullptr;                              // pull, M_RECORD pass: where the input state goes
    // pull: boxes in flight per CTA (1 or 2) for passes without [0] and with [1] observables; FP32
    // defaults from measurements on GB300: FP32 depth 1 (3 CTAs per SM within 80 registers) with
    // and without observables; FP64 depth 2
    int stages[2] = {2, 2};
    // pull: tile width (32 or 64 columns) of the step passes without [0] and with [1] observables;
    // 64 only in FP32; chosen by lbm_autotune_tiles
    int width[2] = {32, 32};
    // the lattices of a batch (one entry for a single lattice): host and device copies
    std::vector<InstGeom> inst;
    InstGeom* inst_d = nullptr;
    std::vector<char> drive_set;  // lattice's drive set by lbm_set_instance_drive
    int ntz_all = 0;              // pull: tile rows of all lattices
    int prows = 0;                // pull: padded rows of a population plane
    double* host_out = nullptr; // pinned
    StepConst<float> c32{};
    StepConst<double> c64{};
    double rho_ref[2] = {0.0, 0.0};
    bool have_params = false, have_fields = false;
    int observe_every = 0;
    long long samples = 0;  // states accumulated into the time sums since the last reset
    long long step = 0;
    long long launches = 0;
    // [parity][observe][first launch folds no pending reduction (0), one without (1) / with (2)
    // accumulation into the time sums][counter of the first launch]
    cudaGraphExec_t graph[2][2][3][2] = {};
    int graph_steps = 16;
    bool profiling = false;
    std::vector<cudaEvent_t> ev;  // pairs around step-kernel launches
    size_t ev_used = 0;
    std::vector<cudaEvent_t> aev;  // adjoint: three pairs per step, around its kernels
    size_t aev_used = 0;
    unsigned serial = 0;           // this context's number among the contexts of the process
    unsigned snap_seq = 0;         // snapshots written so far
    std::map<const void*, SnapTail> snaps;  // tails of this context's latest snapshots, by address
    std::vector<const void*> snap_order;    // their addresses, oldest first (bounds the map)
    cudaEvent_t tev[64] = {};      // asynchronous reads: an event per ticket (ring)
    double* rec_dst = nullptr;     // lbm_step_read: where the next launch's folded sample goes
    long long tickets = 0;         // tickets issued
    std::string err;
};

static std::string g_create_error;

static int fail(lbm_ctx* c, int code, const char* fmt, ...) {
    char buf[512];
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(buf, sizeof buf, fmt, ap);
    va_end(ap);
    if (c)
        c->err = buf;
    else
        g_create_error = buf;
    return code;
}

#define CK(call)                                                                                  \
    do {                                                                                          \
        cudaError_t e_ = (call);                                                                  \
        if (e_ != cudaSuccess)                                                                    \
            return fail(c, e_ == cudaErrorMemoryAllocation ? LBM_ENOMEM : LBM_ECUDA, "%s: %s (%s:%d)", #call, \
                        cudaGetErrorString(e_), __FILE__, __LINE__);                              \
    } while (0)

static Batch batch(const lbm_ctx* c) { return Batch{c->inst_d, (int)c->inst.size(), c->ntz_all}; }

// Device copy of the lattices' table (geometry and drives).
static cudaError_t upload_inst(lbm_ctx* c) {
    return cudaMemcpyAsync(c->inst_d, c->inst.data(), c->inst.size() * sizeof(InstGeom), cudaMemcpyHostToDevice,
                           c->stream);
}

static void refresh_const(lbm_ctx* c) {
    fill_step_const<float>(c->c32, c->p, c->d.nx, c->d.nz, c->pitch, c->plane, c->d.n_species, c->d.z_boundary,
                           c->rho_ref);
    fill_step_const<double>(c->c64, c->p, c->d.nx, c->d.nz, c->pitch, c->plane, c->d.n_species, c->d.z_boundary,
                            c->rho_ref);
    for (size_t i = 0; i < c->inst.size(); ++i)  // the parameters' drive, where no lattice drive is set
        if (!c->drive_set[i]) {
            set_inst_drive(c->inst[i], c->p.body_force, c->p.wall_u[0], c->p.wall_u[1]);
        }
}

static void drop_graphs(lbm_ctx* c) {
    for (auto& pr : c->graph)
        for (auto& po : pr)
            for (auto& pf : po)
                for (auto& g : pf)
                    if (g) {
                        cudaGraphExecDestroy(g);
                        g = nullptr;
                    }
}

static size_t obs_bytes(const lbm_ctx* c) {
    return (size_t)(obs_len(c->d.nx, c->d.nz) + 5LL * reduce_blocks(c->d.nx, c->d.nz)) * sizeof(double);
}

// ---------------------------------------------------------------------------------------
// Validation (host only)
// ---------------------------------------------------------------------------------------
extern "C" void lbm_default_desc(lbm_desc* d) {
    if (!d) return;
    memset(d, 0, sizeof *d);
    d->nx = d->nz = 64;
    d->n_species = 1;
    d->precision = LBM_FP64;
    d->z_boundary = LBM_PERIODIC;
    d->kernel = LBM_KERNEL_AUTO;
}

extern "C" void lbm_default_params(lbm_params* p) {
    if (!p) return;
    memset(p, 0, sizeof *p);
    p->tau[0] = p->tau[1] = 1.0;
    p->rho0[0] = p->rho0[1] = 1.0;
    p->weight_norm = 1.0 / 3.0;
    p->rho_ref[0] = p->rho_ref[1] = -1.0;
}

static int check_desc(lbm_ctx* c, const lbm_desc* d) {
    if (!d) return fail(c, LBM_EINVAL, "desc is NULL");
    if (d->nx < 1 || d->nz < 1 || d->nx > 65536 || d->nz > 65536)
        return fail(c, LBM_EINVAL, "nx, nz must be in [1, 65536] (got %d x %d)", d->nx, d->nz);
    if ((long long)d->nx * d->nz > (1LL << 30)) return fail(c, LBM_EINVAL, "nx * nz exceeds 2^30");
    if (d->n_species != 1 && d->n_species != 2) return fail(c, LBM_EINVAL, "n_species must be 1 or 2");
    if (d->precision != LBM_FP64 && d->precision != LBM_FP32) return fail(c, LBM_EINVAL, "unknown precision");
    if (d->z_boundary != LBM_PERIODIC && d->z_boundary != LBM_BOUNCEBACK)
        return fail(c, LBM_EINVAL, "unknown z boundary");
    if (d->kernel < LBM_KERNEL_AUTO || d->kernel > LBM_KERNEL_PULL) return fail(c, LBM_EINVAL, "unknown kernel");
    if (d->rows_per_warp < 0 || d->rows_per_warp > 65536) return fail(c, LBM_EINVAL, "rows_per_warp out of range");
    if (d->tile_rows != 0 && d->tile_rows != 8 && d->tile_rows != 16)
        return fail(c, LBM_EINVAL, "tile_rows must be 0, 8 or 16");
    if (d->device < 0) return fail(c, LBM_EINVAL, "negative device ordinal");
    if (d->n_instances < 0 || d->n_instances > 4096) return fail(c, LBM_EINVAL, "n_instances must be in [0, 4096]");
    if (d->n_instances > 1) {
        if (!d->inst_nz) return fail(c, LBM_EINVAL, "inst_nz is NULL");
        long long sum = 0;
        for (int i = 0; i < d->n_instances; ++i) {
            if (d->inst_nz[i] < 1) return fail(c, LBM_EINVAL, "inst_nz[%d] = %d is not >= 1", i, d->inst_nz[i]);
            sum += d->inst_nz[i];
        }
        if (sum != d->nz) return fail(c, LBM_EINVAL, "nz (%d) must equal the sum of inst_nz (%lld)", d->nz, sum);
        if (d->z_boundary != LBM_BOUNCEBACK) return fail(c, LBM_EINVAL, "a batch needs LBM_BOUNCEBACK walls");
        if (d->kernel != LBM_KERNEL_AUTO && d->kernel != LBM_KERNEL_PULL)
            return fail(c, LBM_EINVAL, "a batch runs on the PULL kernel");
    }
    return LBM_OK;
}

static int check_params(lbm_ctx* c, const lbm_params* p, int ns) {
    if (!p) return fail(c, LBM_EINVAL, "params is NULL");
    for (int s = 0; s < ns; ++s) {
        if (!(p->tau[s] > 0.5) || !std::isfinite(p->tau[s])) return fail(c, LBM_EINVAL, "tau[%d] must be > 1/2", s);
        if (!std::isfinite(p->G1[s]) || !std::isfinite(p->G2[s])) return fail(c, LBM_EINVAL, "G1/G2 not finite");
        if (p->psi_form == LBM_PSI_EXP && !(p->rho0[s] > 0.0 && std::isfinite(p->rho0[s])))
            return fail(c, LBM_EINVAL, "rho0[%d] must be > 0", s);
        if (!std::isfinite(p->rho_ref[s])) return fail(c, LBM_EINVAL, "rho_ref not finite");
    }
    if (p->psi_form != LBM_PSI_EXP && p->psi_form != LBM_PSI_RHO) return fail(c, LBM_EINVAL, "unknown psi form");
    if (p->weight_preset != LBM_WEIGHTS_PAPER && p->weight_preset != LBM_WEIGHTS_CHEM09)
        return fail(c, LBM_EINVAL, "unknown weight preset");
    if (p->psi_wall != LBM_WALL_MIRROR && p->psi_wall != LBM_WALL_ZERO) return fail(c, LBM_EINVAL, "unknown psi_wall");
    if (!(p->weight_norm > 0.0) || !std::isfinite(p->weight_norm)) return fail(c, LBM_EINVAL, "weight_norm must be > 0");
    if (!std::isfinite(p->G_AB) || !std::isfinite(p->body_force) || !std::isfinite(p->wall_u[0]) ||
        !std::isfinite(p->wall_u[1]))
        return fail(c, LBM_EINVAL, "G_AB, body_force, wall_u must be finite");
    return LBM_OK;
}

extern "C" int lbm_validate_desc(const lbm_desc* d) { return check_desc(nullptr, d); }
extern "C" int lbm_validate_params(const lbm_params* p, int n_species) {
    if (n_species != 1 && n_species != 2) return fail(nullptr, LBM_EINVAL, "n_species must be 1 or 2");
    return check_params(nullptr, p, n_species);
}

// ---------------------------------------------------------------------------------------
// Creation
// ---------------------------------------------------------------------------------------
static void release(lbm_ctx* c) {
    if (!c) return;
    if (c->d.device >= 0) cudaSetDevice(c->d.device);
    drop_graphs(c);
    for (cudaEvent_t e : c->ev) cudaEventDestroy(e);
    c->ev.clear();
    for (cudaEvent_t e : c->aev) cudaEventDestroy(e);
    c->aev.clear();
    for (cudaEvent_t& e : c->tev)
        if (e) cudaEventDestroy(e);
    void* ptrs[] = {c->f_raw[0],   c->f_raw[1], c->part_row[0], c->part_row[1], c->part_col[0],
                    c->part_col[1], c->sched,   c->ticket,      c->flag,        c->out,
                    c->avg,         c->staging, c->fexport,     c->gfield,      c->inst_d,
                    c->adj_scratch, c->adj_lam,    c->dcheck};
    for (void* p : ptrs)
        if (p) cudaFree(p);
    if (c->host_out) cudaFreeHost(c->host_out);
    if (c->own_stream && c->stream) cudaStreamDestroy(c->stream);
}

// Rows per warp: the smallest chunk height for which every warp of the grid is resident at
// once (one wave), so no SM idles in a tail and the 4-row prologue per chunk stays small.
static SweepGeom sweep_geom(const lbm_ctx* c, int resident_warps) {
    SweepGeom g;
    g.nstrips = (c->d.nx + STRIP_W - 1) / STRIP_W;
    long long hz;
    if (c->d.rows_per_warp > 0) {
        hz = c->d.rows_per_warp;
    } else {
        const long long target = resident_warps > 0 ? resident_warps : 152LL * 8;
        hz = ((long long)c->d.nz * g.nstrips + target - 1) / target;
        if (hz < 2) hz = 2;
    }
    if (hz > c->d.nz) hz = c->d.nz;
    g.hz = (int)hz;
    g.nchunks = (c->d.nz + g.hz - 1) / g.hz;
    return g;
}

extern "C" int lbm_create(lbm_ctx** out, const lbm_desc* d) {
    g_create_error.clear();
    if (!out) return fail(nullptr, LBM_EINVAL, "out is NULL");
    *out = nullptr;
    int rc = check_desc(nullptr, d);
    if (rc) return rc;
    lbm_ctx* c = new (std::nothrow) lbm_ctx();
    if (!c) return fail(nullptr, LBM_ENOMEM, "host allocation failed");
    c->d = *d;
    c->serial = ++g_ctx_serial;
    lbm_default_params(&c->p);
    auto bail = [&](int code) {
        g_create_error = c->err;
        release(c);
        delete c;
        return code;
    };
#define CKC(call)                                                                                          \
    do {                                                                                                   \
        cudaError_t e_ = (call);                                                                           \
        if (e_ != cudaSuccess)                                                                             \
            return bail(fail(c, e_ == cudaErrorMemoryAllocation ? LBM_ENOMEM : LBM_ECUDA, "%s: %s", #call, \
                             cudaGetErrorString(e_)));                                                     \
    } while (0)
    int ndev = 0;
    CKC(cudaGetDeviceCount(&ndev));
    if (d->device >= ndev) return bail(fail(c, LBM_EINVAL, "device %d not present (%d devices)", d->device, ndev));
    CKC(cudaSetDevice(d->device));
    cudaDeviceProp prop;
    CKC(cudaGetDeviceProperties(&prop, d->device));
    c->nsm = prop.multiProcessorCount;
    if (d->stream) {
        c->stream = (cudaStream_t)d->stream;
    } else {
        CKC(cudaStreamCreateWithFlags(&c->stream, cudaStreamNonBlocking));
        c->own_stream = true;
    }
    const int nx = d->nx, nz = d->nz, ns = d->n_species;
    c->esize = d->precision == LBM_FP64 ? sizeof(double) : sizeof(float);
    if (d->precision == LBM_FP32) c->stages[0] = c->stages[1] = 1;
    c->kernel = d->kernel == LBM_KERNEL_AUTO ? LBM_KERNEL_PULL : d->kernel;
    c->pull = c->kernel == LBM_KERNEL_PULL;
    {  // the lattices: rows stacked in order, each with its own ghost rows in the planes
        const int ni = d->n_instances > 1 ? d->n_instances : 1;
        c->inst.assign(ni, InstGeom{});
        c->drive_set.assign(ni, 0);
        int zrow = 0, prow = 0, trow = 0;
        for (int i = 0; i < ni; ++i) {
            InstGeom& g = c->inst[i];
            g.nz = ni > 1 ? d->inst_nz[i] : nz;
            g.zrow0 = zrow;
            g.prow0 = prow;
            g.trow0 = trow;
            g.ntz = (g.nz + 7) / 8;
            zrow += g.nz;
            prow += g.nz + 2 * PULL_GZ;
            trow += g.ntz;
        }
        c->ntz_all = trow;
        c->prows = prow;
        CKC(cudaMalloc(&c->inst_d, ni * sizeof(InstGeom)));
    }
    if (c->pull) {  // ghost columns and rows around every lattice; 128-byte rows
        c->pitch = (nx + 2 * PULL_GX + 31) / 32 * 32;
        c->plane = (long long)c->prows * c->pitch;
    } else {
        c->pitch = (nx + 31) / 32 * 32;
        c->plane = (long long)nz * c->pitch;
    }
    c->tile_rows = c->pull || d->tile_rows == 0 ? 8 : d->tile_rows;
    const size_t fbytes = (size_t)ns * 9 * c->plane * c->esize;
    // pull layout: shift the origin so that every row's first lattice column (padded column
    // PULL_GX) starts a 128-byte line; the shift keeps the 16-byte alignment tensor maps need
    const size_t shift = c->pull ? (128 - (PULL_GX * c->esize) % 128) % 128 : 0;
    for (int b = 0; b < 2; ++b) {
        CKC(cudaMalloc(&c->f_raw[b], fbytes + 128));
        c->f[b] = static_cast<char*>(c->f_raw[b]) + shift;
    }
    CKC(cudaMemsetAsync(c->f[0], 0, fbytes, c->stream));
    CKC(cudaMemsetAsync(c->f[1], 0, fbytes, c->stream));
    // fused geometry and partial-sum groups
    {
        const bool f64 = d->precision == LBM_FP64;
        const int rw = f64 ? fused_resident_warps<double>(ns, M_WRITE, c->nsm)
                           : fused_resident_warps<float>(ns, M_WRITE, c->nsm);
        const int ro = f64 ? fused_resident_warps<double>(ns, M_WRITE | M_OBS, c->nsm)
                           : fused_resident_warps<float>(ns, M_WRITE | M_OBS, c->nsm);
        if (rw <= 0 || ro <= 0) return bail(fail(c, LBM_ECUDA, "occupancy query of the step kernel failed"));
        c->geom = sweep_geom(c, rw);
        c->geom_obs = sweep_geom(c, ro);
    }
    const int tx = (nx + TPX - 1) / TPX, tz = (nz + std::min(TPZ, 8) - 1) / std::min(TPZ, 8);
    const long long rows_parts = std::max(c->geom_obs.nstrips, tx);
    const long long col_parts = std::max(std::max(std::max(c->geom_obs.nchunks, c->geom.nchunks), tz), c->ntz_all);
    for (int b = 0; b < 2; ++b) {
        CKC(cudaMalloc(&c->part_row[b], (size_t)rows_parts * nz * NQR * c->esize));
        CKC(cudaMalloc(&c->part_col[b], (size_t)col_parts * nx * NQC * c->esize));
    }
    CKC(cudaMalloc(&c->sched, 4 * sizeof(unsigned)));
    CKC(cudaMemsetAsync(c->sched, 0, 4 * sizeof(unsigned), c->stream));
    CKC(cudaMalloc(&c->ticket, sizeof(unsigned)));
    CKC(cudaMalloc(&c->flag, sizeof(int)));
    // observables: obs_len entries, then the reduction's block partials of the scalars
    const size_t olen = (size_t)(obs_len(nx, nz) + 5LL * reduce_blocks(nx, nz)) * sizeof(double);
    // each followed by room for the trailer of an asynchronous read (lbm_observables_enqueue)
    CKC(cudaMalloc(&c->out, olen + 64));
    CKC(cudaMalloc(&c->avg, olen + 64));
    CKC(cudaMalloc(&c->staging, (size_t)(ns + 2) * nx * nz * sizeof(double)));
    CKC(cudaMalloc(&c->dcheck, DCHECK_DOUBLES * sizeof(double)));
    CKC(cudaMallocHost(&c->host_out, olen));
    CKC(cudaMemsetAsync(c->ticket, 0, sizeof(unsigned), c->stream));
    CKC(cudaMemsetAsync(c->flag, 0, sizeof(int), c->stream));
    CKC(cudaMemsetAsync(c->avg, 0, olen, c->stream));
    if (c->kernel == LBM_KERNEL_TWO_PASS) {
        c->ghost.gpitch = (nx + 2 * GX + 3) / 4 * 4;  // 16-byte rows for the TMA descriptor
        c->ghost.gplane = (long long)(nz + 4) * c->ghost.gpitch;
        CKC(cudaMalloc(&c->gfield, (size_t)2 * ns * c->ghost.gplane * c->esize));
        CKC(cudaMemsetAsync(c->gfield, 0, (size_t)2 * ns * c->ghost.gplane * c->esize, c->stream));
        if (make_field_tmap(c->tmap, c->gfield, (int)c->esize, ns, nz, c->ghost) != 0)
            return bail(fail(c, LBM_ECUDA, "cuTensorMapEncodeTiled failed for the two-pass field planes"));
    }
    if (c->pull) {
        for (int b = 0; b < 2; ++b) {
            if (make_pop_tmap(c->pmap_in[b], c->f[b], (int)c->esize, ns, c->prows, c->pitch, c->plane, 32) != 0)
                return bail(fail(c, LBM_ECUDA, "cuTensorMapEncodeTiled failed for the population buffers"));
            if (d->precision == LBM_FP32 &&
                make_pop_tmap(c->pmap_wide[b], c->f[b], (int)c->esize, ns, c->prows, c->pitch, c->plane, 64) != 0)
                return bail(fail(c, LBM_ECUDA, "cuTensorMapEncodeTiled failed for the population buffers"));
        }
        const int per = d->z_boundary == LBM_PERIODIC ? M_PERIODIC : 0;
        const int modes[5] = {M_WRITE, M_WRITE | M_OBS | per, M_OBS | per, M_FIELDS, M_WRITE | M_RECORD};
        for (int m : modes)
            for (int st = 1; st <= 2; ++st) {
                const int nb = d->precision == LBM_FP64 ? pull_blocks_per_sm<double>(ns, m, st, 32)
                                                        : pull_blocks_per_sm<float>(ns, m, st, 32);
                if (nb < 1) return bail(fail(c, LBM_ECUDA, "occupancy query of the pull kernel failed"));
                c->pull_grid[m][st - 1][0] = nb * c->nsm;
                if (d->precision == LBM_FP32 && (m == M_WRITE || m == (M_WRITE | M_OBS | per))) {
                    const int nw = pull_blocks_per_sm<float>(ns, m, st, 64);
                    if (nw < 1) return bail(fail(c, LBM_ECUDA, "occupancy query of the pull kernel failed"));
                    c->pull_grid[m][st - 1][1] = nw * c->nsm;
                }
            }
    }
    refresh_const(c);
    CKC(upload_inst(c));
    CKC(cudaStreamSynchronize(c->stream));
#undef CKC
    *out = c;
    return LBM_OK;
}

extern "C" void lbm_destroy(lbm_ctx* c) {
    if (!c) return;
    if (c->stream) cudaStreamSynchronize(c->stream);
    release(c);
    delete c;
}

extern "C" int lbm_set_params(lbm_ctx* c, const lbm_params* p) {
    if (!c) return LBM_EINVAL;
    int rc = check_params(c, p, c->d.n_species);
    if (rc) return rc;
    c->p = *p;
    c->have_params = true;
    std::fill(c->drive_set.begin(), c->drive_set.end(), 0);
    refresh_const(c);
    CK(upload_inst(c));
    drop_graphs(c);
    return LBM_OK;
}

extern "C" int lbm_set_instance_drive(lbm_ctx* c, int i, double body_force, double wall_u_bottom,
                                      double wall_u_top) {
    if (!c) return LBM_EINVAL;
    if (i < 0 || i >= (int)c->inst.size()) return fail(c, LBM_EINVAL, "lattice %d not in the batch", i);
    if (!std::isfinite(body_force) || !std::isfinite(wall_u_bottom) || !std::isfinite(wall_u_top))
        return fail(c, LBM_EINVAL, "drive values must be finite");
    CK(cudaSetDevice(c->d.device));
    if (!c->pull) {  // one lattice on another kernel: the drive lives in the step constants
        c->p.body_force = body_force;
        c->p.wall_u[0] = wall_u_bottom;
        c->p.wall_u[1] = wall_u_top;
        refresh_const(c);
        drop_graphs(c);
    }
    set_inst_drive(c->inst[i], body_force, wall_u_bottom, wall_u_top);
    c->drive_set[i] = 1;
    CK(upload_inst(c));  // the kernels read the table at run time: captured graphs stay valid
    return LBM_OK;
}

// ---------------------------------------------------------------------------------------
// Step kernels
// ---------------------------------------------------------------------------------------
static ObsPtrs obs_ptrs(const lbm_ctx* c, int buf) {
    ObsPtrs O;
    O.part_row = c->part_row[buf];
    O.part_col = c->part_col[buf];
    O.fields = c->staging;
    O.flag = c->flag;
    return O;
}

// The reduction kernel over the partial sums in part_*[buf] (of a pass at parity buf).
static cudaError_t reduce_now(lbm_ctx* c, int buf, bool accumulate) {
    const bool sweep = c->kernel == LBM_KERNEL_SWEEP;
    const int tzrows = c->kernel == LBM_KERNEL_TWO_PASS ? TPZ : c->tile_rows;
    const int nxp = sweep ? c->geom_obs.nstrips : (c->d.nx + TPX - 1) / TPX;
    const int nzp = sweep ? c->geom_obs.nchunks : c->pull ? c->ntz_all : (c->d.nz + tzrows - 1) / tzrows;
    const long long ol = obs_len(c->d.nx, c->d.nz);
    const int ni = (int)c->inst.size();
    c->launches += 1;
    return launch_reduce((int)c->esize, obs_ptrs(c, buf), nxp, nzp, c->d.nx, c->d.nz, c->d.z_boundary, c->ticket,
                         c->out, c->avg, c->out + ol, c->avg + ol, accumulate ? 1 : 0, false,
                         ni > 1 ? c->inst_d : nullptr, ni, c->stream);
}

// A reduction left pending by the pull kernel, run now (before the host reads or resets the
// observable buffers).
static cudaError_t flush_pending(lbm_ctx* c) {
    if (!c->pending) return cudaSuccess;
    c->pending = false;
    return reduce_now(c, c->pending_buf, c->pending_acc);
}

// One pass of the step kernel over the state in f[cur] (mode: M_WRITE into f[cur^1],
// M_OBS partial sums into part_*[cur], M_FIELDS per-site fields), plus the reduction when
// `reduce`.  With the pull kernel and `defer` the reduction is left pending and folded into the
// next pull launch; any pending reduction is folded into this launch.
static cudaError_t enqueue_pass(lbm_ctx* c, int cur, int mode, bool reduce, bool accumulate, bool defer) {
    const ObsPtrs O = obs_ptrs(c, cur);
    cudaError_t e;
    Fold Rd{};
    if (c->pull && c->pending) {
        if (c->pending_buf == cur && (mode & M_OBS)) {
            e = flush_pending(c);  // this pass would overwrite the pending partial sums
            if (e != cudaSuccess) return e;
        } else {
            const long long ol = obs_len(c->d.nx, c->d.nz);
            Rd.part_row = c->part_row[c->pending_buf];
            Rd.part_col = c->part_col[c->pending_buf];
            Rd.out = c->out;
            Rd.bpart = c->out + ol;
            Rd.nxpart = (c->d.nx + TPX - 1) / TPX;
            Rd.nzpart = c->ntz_all;
            if (c->rec_dst && c->pending_acc) {  // the sample goes into a record of its own
                Rd.avg = c->rec_dst;
                Rd.bavg = c->rec_dst + ol;
                Rd.accumulate = 2;
            } else {
                Rd.avg = c->avg;
                Rd.bavg = c->avg + ol;
                Rd.accumulate = c->pending_acc ? 1 : 0;
            }
            Rd.enabled = 1;
            // the reciprocals in the populations' precision, as the reduction kernel takes them
            Rd.inx = c->esize == 4 ? (double)(1.0f / (float)c->d.nx) : 1.0 / c->d.nx;
            Rd.inz = c->esize == 4 ? (double)(1.0f / (float)c->d.nz) : 1.0 / c->d.nz;
            c->pending = false;
        }
    }
    const bool timed = c->profiling && (mode & M_WRITE);
    if (timed) {
        if (c->ev_used + 2 > c->ev.size()) {
            for (int k = 0; k < 64; ++k) {
                cudaEvent_t ev;
                e = cudaEventCreate(&ev);
                if (e != cudaSuccess) return e;
                c->ev.push_back(ev);
            }
        }
        e = cudaEventRecord(c->ev[c->ev_used], c->stream);
        if (e != cudaSuccess) return e;
    }
    const bool twopass = c->kernel == LBM_KERNEL_TWO_PASS && (mode & M_WRITE);
    const int tpx = (c->d.nx + TPX - 1) / TPX;
    const int tzrows = twopass ? TPZ : c->tile_rows;
    const int tpz = (c->d.nz + tzrows - 1) / tzrows;
    if (twopass) {
        // K1: densities and pseudopotentials into the ghost-padded planes; K2: collide and push
        if (c->d.precision == LBM_FP64) {
            e = launch_density<double>(c->d.n_species, (const double*)c->f[cur], (double*)c->gfield, c->c64, c->ghost,
                                       c->stream);
            if (e == cudaSuccess)
                e = launch_twopass<double>(c->d.n_species, mode, (const double*)c->f[cur], (double*)c->f[cur ^ 1],
                                           (const double*)c->gfield, c->c64, c->ghost, c->tmap, O, tpx, tpz, c->stream);
        } else {
            e = launch_density<float>(c->d.n_species, (const float*)c->f[cur], (float*)c->gfield, c->c32, c->ghost,
                                      c->stream);
            if (e == cudaSuccess)
                e = launch_twopass<float>(c->d.n_species, mode, (const float*)c->f[cur], (float*)c->f[cur ^ 1],
                                          (const float*)c->gfield, c->c32, c->ghost, c->tmap, O, tpx, tpz, c->stream);
        }
        c->launches += 1;
    } else if (c->pull) {
        const Batch B = batch(c);
        // observing passes on periodic lattices run the build without wall logic (fewer
        // instructions and registers); the others run the general build, which fits the
        // depth-1 register budget without spills
        const int pm = mode | (c->d.z_boundary == LBM_PERIODIC && (mode & M_OBS) ? M_PERIODIC : 0);
        const int cls = (mode & M_OBS) ? 1 : 0;
        const int stg = c->stages[cls];
        // the tuned width applies to the step passes (write, observing or not); other passes run 32
        const bool wide = c->width[cls] == 64 && c->d.precision == LBM_FP32 && c->pull_grid[pm][stg - 1][1] > 0;
        const void* tin = wide ? c->pmap_wide[cur] : c->pmap_in[cur];
        const int grid = c->pull_grid[pm][stg - 1][wide ? 1 : 0];
        if (c->d.precision == LBM_FP64)
            e = launch_pull<double>(c->d.n_species, pm, stg, 32, tin, (double*)c->f[cur ^ 1], c->c64, O,
                                    Rd, c->sched, c->sched_set, B, grid, c->stream, (double*)c->rec);
        else
            e = launch_pull<float>(c->d.n_species, pm, stg, wide ? 64 : 32, tin, (float*)c->f[cur ^ 1], c->c32, O,
                                   Rd, c->sched, c->sched_set, B, grid, c->stream, (float*)c->rec);
        if (e == cudaSuccess) c->sched_set ^= 1;
    } else if (c->kernel == LBM_KERNEL_SWEEP) {
        const SweepGeom& G = (mode & M_OBS) ? c->geom_obs : c->geom;
        if (c->d.precision == LBM_FP64)
            e = launch_fused<double>(c->d.n_species, mode, (const double*)c->f[cur], (double*)c->f[cur ^ 1], c->c64, G,
                                     O, c->stream);
        else
            e = launch_fused<float>(c->d.n_species, mode, (const float*)c->f[cur], (float*)c->f[cur ^ 1], c->c32, G, O,
                                    c->stream);
    } else {
        if (c->d.precision == LBM_FP64)
            e = launch_tile<double>(c->d.n_species, mode, c->tile_rows, (const double*)c->f[cur], (double*)c->f[cur ^ 1],
                                    c->c64, O, c->stream);
        else
            e = launch_tile<float>(c->d.n_species, mode, c->tile_rows, (const float*)c->f[cur], (float*)c->f[cur ^ 1],
                                   c->c32, O, c->stream);
    }
    c->launches += 1;
    if (e != cudaSuccess) return e;
    if (timed) {
        e = cudaEventRecord(c->ev[c->ev_used + 1], c->stream);
        if (e != cudaSuccess) return e;
        c->ev_used += 2;
    }
    if (reduce) {
        if (c->pull && defer) {
            c->pending = true;
            c->pending_buf = cur;
            c->pending_acc = accumulate;
        } else {
            e = reduce_now(c, cur, accumulate);
        }
        if (accumulate) c->samples += 1;
    }
    return e;
}

static bool observe_now(const lbm_ctx* c, long long step) {
    return c->observe_every > 0 && step % c->observe_every == 0;
}

extern "C" int lbm_step(lbm_ctx* c, int nsteps) {
    if (!c || nsteps < 0) return c ? fail(c, LBM_EINVAL, "nsteps < 0") : LBM_EINVAL;
    if (!c->have_fields) return fail(c, LBM_EINVAL, "lbm_set_fields has not been called");
    CK(cudaSetDevice(c->d.device));
    int left = nsteps;
    const int G = c->graph_steps;
    const bool graphable = !c->profiling && (c->observe_every == 0 || c->observe_every == 1);
    while (left > 0) {
        if (graphable && left >= G) {
            const int ob = c->observe_every == 1 ? 1 : 0;
            const int ff = c->pull && c->pending ? (c->pending_acc ? 2 : 1) : 0;
            cudaGraphExec_t& ge = c->graph[c->cur][ob][ff][c->sched_set];
            if (!ge) {
                cudaGraph_t g = nullptr;
                CK(cudaStreamBeginCapture(c->stream, cudaStreamCaptureModeThreadLocal));
                const long long saved = c->launches, saved_samples = c->samples;
                const bool saved_pending = c->pending, saved_acc = c->pending_acc;
                const int saved_buf = c->pending_buf, saved_set = c->sched_set;
                cudaError_t e = cudaSuccess;
                for (int i = 0; i < G && e == cudaSuccess; ++i)
                    e = enqueue_pass(c, (c->cur + i) & 1, M_WRITE | (ob ? M_OBS : 0), ob, ob, true);
                cudaError_t e2 = cudaStreamEndCapture(c->stream, &g);
                c->launches = saved;
                c->samples = saved_samples;
                c->pending = saved_pending;
                c->pending_acc = saved_acc;
                c->pending_buf = saved_buf;
                c->sched_set = saved_set;  // G is even: a replay leaves the counter of the next launch as it was
                CK(e);
                CK(e2);
                e = cudaGraphInstantiate(&ge, g, 0);
                cudaGraphDestroy(g);
                CK(e);
            }
            CK(cudaGraphLaunch(ge, c->stream));
            c->launches += (long long)G * (ob && !c->pull ? 2 : 1);
            if (ob) c->samples += G;
            if (c->pull) {  // the last step's reduction is pending; an earlier one was folded in
                c->pending = ob;
                c->pending_acc = ob;
                c->pending_buf = c->cur ^ 1;  // parity of the graph's last launch (G is even)
            }
            c->step += G;  // G is even: the parity of cur is unchanged
            left -= G;
            continue;
        }
        const bool ob = observe_now(c, c->step);
        CK(enqueue_pass(c, c->cur, M_WRITE | (ob ? M_OBS : 0), ob, ob, true));
        c->cur ^= 1;
        c->step += 1;
        left -= 1;
    }
    return LBM_OK;
}

extern "C" int lbm_set_observe(lbm_ctx* c, int every) {
    if (!c) return LBM_EINVAL;
    if (every < 0) return fail(c, LBM_EINVAL, "every must be >= 0");
    CK(cudaSetDevice(c->d.device));
    CK(flush_pending(c));  // its sample belongs to the sums being cleared
    c->observe_every = every;
    c->samples = 0;
    CK(cudaMemsetAsync(c->avg, 0, obs_bytes(c), c->stream));
    return LBM_OK;
}

// ---------------------------------------------------------------------------------------
// Fields
// ---------------------------------------------------------------------------------------
extern "C" int lbm_set_fields(lbm_ctx* c, const double* rho, const double* u, int where) {
    if (!c) return LBM_EINVAL;
    if (!rho) return fail(c, LBM_EINVAL, "rho is NULL");
    if (where != LBM_HOST && where != LBM_DEVICE) return fail(c, LBM_EINVAL, "where must be LBM_HOST or LBM_DEVICE");
    CK(cudaSetDevice(c->d.device));
    const Batch B = batch(c);
    const int ns = c->d.n_species;
    const long long n = (long long)c->d.nx * c->d.nz;
    // the densities into the staging buffer, checked and summed there (the reference densities
    // need the sums on the host: one small read-back)
    const cudaMemcpyKind kind = where == LBM_HOST ? cudaMemcpyHostToDevice : cudaMemcpyDeviceToDevice;
    CK(cudaMemcpyAsync(c->staging, rho, (size_t)ns * n * sizeof(double), kind, c->stream));
    CK(launch_density_check(c->staging, n, ns, c->dcheck, c->stream));
    double chk[3];
    CK(cudaMemcpyAsync(chk, c->dcheck, sizeof chk, cudaMemcpyDeviceToHost, c->stream));
    CK(cudaStreamSynchronize(c->stream));
    unsigned long long bad;
    memcpy(&bad, &chk[2], sizeof bad);
    if (bad != ~0ull) {
        double v = 0.0;
        CK(cudaMemcpy(&v, c->staging + bad, sizeof v, cudaMemcpyDeviceToHost));
        return fail(c, LBM_EINVAL, "rho[%d][%lld] = %g is not > 0", (int)(bad / n), (long long)(bad % n), v);
    }
    for (int s = 0; s < ns; ++s)
        c->rho_ref[s] = c->d.precision == LBM_FP64 ? 0.0 : (c->p.rho_ref[s] >= 0.0 ? c->p.rho_ref[s] : chk[s] / n);
    const double* du = nullptr;
    if (u) {
        CK(cudaMemcpyAsync(c->staging + ns * n, u, (size_t)2 * n * sizeof(double), kind, c->stream));
        du = c->staging + ns * n;
    }
    refresh_const(c);
    drop_graphs(c);
    c->cur = 0;
    if (c->d.precision == LBM_FP64) {
        CK(launch_init<double>(ns, (double*)c->f[0], c->staging, du, c->c64, c->pull ? &B : nullptr, c->stream));
        if (c->pull) CK(launch_pull_images<double>(ns, (double*)c->f[0], c->c64, B, c->stream));
    } else {
        CK(launch_init<float>(ns, (float*)c->f[0], c->staging, du, c->c32, c->pull ? &B : nullptr, c->stream));
        if (c->pull) CK(launch_pull_images<float>(ns, (float*)c->f[0], c->c32, B, c->stream));
    }
    c->launches += c->pull ? 2 : 1;
    CK(cudaMemsetAsync(c->flag, 0, sizeof(int), c->stream));
    CK(cudaMemsetAsync(c->avg, 0, obs_bytes(c), c->stream));
    c->samples = 0;
    c->pending = false;  // partial sums of the replaced state
    CK(cudaStreamSynchronize(c->stream));
    c->step = 0;
    c->have_fields = true;
    return LBM_OK;
}

extern "C" int lbm_set_populations(lbm_ctx* c, const double* f, int where) {
    if (!c) return LBM_EINVAL;
    if (!f) return fail(c, LBM_EINVAL, "f is NULL");
    if (where != LBM_HOST && where != LBM_DEVICE) return fail(c, LBM_EINVAL, "where must be LBM_HOST or LBM_DEVICE");
    CK(cudaSetDevice(c->d.device));
    const Batch B = batch(c);
    const int ns = c->d.n_species;
    const long long n = (long long)c->d.nx * c->d.nz;
    const size_t bytes = (size_t)ns * 9 * n * sizeof(double);
    if (!c->fexport) CK(cudaMalloc(&c->fexport, bytes));
    CK(cudaMemcpyAsync(c->fexport, f, bytes, where == LBM_HOST ? cudaMemcpyHostToDevice : cudaMemcpyDeviceToDevice,
                       c->stream));
    if (c->d.precision == LBM_FP32)
        for (int s = 0; s < ns; ++s)
            if (c->p.rho_ref[s] >= 0.0)
                c->rho_ref[s] = c->p.rho_ref[s];
            else if (!c->have_fields)
                return fail(c, LBM_EINVAL,
                            "FP32 populations need a reference density: set rho_ref >= 0 or call lbm_set_fields first");
    refresh_const(c);
    drop_graphs(c);
    c->cur = 0;
    if (c->d.precision == LBM_FP64) {
        CK(launch_import<double>(ns, (double*)c->f[0], c->fexport, c->c64, c->pull ? &B : nullptr, c->stream));
        if (c->pull) CK(launch_pull_images<double>(ns, (double*)c->f[0], c->c64, B, c->stream));
    } else {
        CK(launch_import<float>(ns, (float*)c->f[0], c->fexport, c->c32, c->pull ? &B : nullptr, c->stream));
        if (c->pull) CK(launch_pull_images<float>(ns, (float*)c->f[0], c->c32, B, c->stream));
    }
    c->launches += c->pull ? 2 : 1;
    CK(cudaMemsetAsync(c->flag, 0, sizeof(int), c->stream));
    CK(cudaMemsetAsync(c->avg, 0, obs_bytes(c), c->stream));
    c->samples = 0;
    c->pending = false;
    CK(cudaStreamSynchronize(c->stream));
    c->step = 0;
    c->have_fields = true;
    return LBM_OK;
}

// A snapshot: the current population buffer in the internal layout, then a 256-byte tail (SnapTail).
static size_t pop_bytes(const lbm_ctx* c) { return (size_t)c->d.n_species * 9 * c->plane * c->esize; }

extern "C" long long lbm_snapshot_bytes(const lbm_ctx* c) { return c ? (long long)(pop_bytes(c) + 256) : -1; }

static SnapTail make_tail(const lbm_ctx* c, unsigned long long tag) {
    SnapTail t{};
    t.rho_ref[0] = c->rho_ref[0];
    t.rho_ref[1] = c->rho_ref[1];
    t.step = c->step;
    t.tag = tag;
    t.nx = c->d.nx;
    t.nz = c->d.nz;
    t.ns = c->d.n_species;
    t.precision = c->d.precision;
    t.n_inst = (int)c->inst.size();
    return t;
}

extern "C" int lbm_snapshot(lbm_ctx* c, void* dst) {
    if (!c) return LBM_EINVAL;
    if (!dst) return fail(c, LBM_EINVAL, "dst is NULL");
    if (!c->have_fields) return fail(c, LBM_EINVAL, "lbm_set_fields has not been called");
    CK(cudaSetDevice(c->d.device));
    CK(cudaMemcpyAsync(dst, c->f[c->cur], pop_bytes(c), cudaMemcpyDeviceToDevice, c->stream));
    const SnapTail t = make_tail(c, (unsigned long long)c->serial << 32 | ++c->snap_seq);
    // pageable source: staged before the call returns
    CK(cudaMemcpyAsync(static_cast<char*>(dst) + pop_bytes(c), &t, sizeof t, cudaMemcpyHostToDevice, c->stream));
    // remembered for lbm_restore_own; the oldest entry goes when the map is full
    if (c->snaps.find(dst) == c->snaps.end()) {
        if (c->snap_order.size() >= SNAP_CACHE_MAX) {
            c->snaps.erase(c->snap_order.front());
            c->snap_order.erase(c->snap_order.begin());
        }
        c->snap_order.push_back(dst);
    }
    c->snaps[dst] = t;
    return LBM_OK;
}

// Makes the populations at src and the tail t the current state (in stream order).
static int restore_from(lbm_ctx* c, const void* src, const SnapTail& t, bool check_tag) {
    CK(cudaMemcpyAsync(c->f[0], src, pop_bytes(c), cudaMemcpyDeviceToDevice, c->stream));
    if (t.rho_ref[0] != c->rho_ref[0] || t.rho_ref[1] != c->rho_ref[1]) {
        c->rho_ref[0] = t.rho_ref[0];
        c->rho_ref[1] = t.rho_ref[1];
        refresh_const(c);
        drop_graphs(c);
    }
    c->cur = 0;
    CK(cudaMemsetAsync(c->flag, 0, sizeof(int), c->stream));
    if (check_tag) {
        CK(launch_snap_check(static_cast<const unsigned long long*>(
                                 static_cast<const void*>(static_cast<const char*>(src) + pop_bytes(c) +
                                                          offsetof(SnapTail, tag))),
                             t.tag, c->flag, c->stream));
        c->launches += 1;
    }
    CK(cudaMemsetAsync(c->avg, 0, obs_bytes(c), c->stream));
    c->samples = 0;
    c->pending = false;
    c->step = t.step;
    c->have_fields = true;
    return LBM_OK;
}

extern "C" int lbm_restore(lbm_ctx* c, const void* src) {
    if (!c) return LBM_EINVAL;
    if (!src) return fail(c, LBM_EINVAL, "src is NULL");
    CK(cudaSetDevice(c->d.device));
    SnapTail t;
    CK(cudaMemcpyAsync(&t, static_cast<const char*>(src) + pop_bytes(c), sizeof t, cudaMemcpyDeviceToHost,
                       c->stream));
    CK(cudaStreamSynchronize(c->stream));
    if (t.nx != c->d.nx || t.nz != c->d.nz || t.ns != c->d.n_species || t.precision != c->d.precision ||
        t.n_inst != (int)c->inst.size() || (t.tag >> 32) == 0)
        return fail(c, LBM_EINVAL, "src holds no snapshot of a context of this shape and precision");
    const int rc = restore_from(c, src, t, false);
    if (rc) return rc;
    CK(cudaStreamSynchronize(c->stream));
    return LBM_OK;
}

extern "C" int lbm_restore_own(lbm_ctx* c, const void* src) {
    if (!c) return LBM_EINVAL;
    if (!src) return fail(c, LBM_EINVAL, "src is NULL");
    const auto known = c->snaps.find(src);
    if (known == c->snaps.end()) return lbm_restore(c, src);
    CK(cudaSetDevice(c->d.device));
    return restore_from(c, src, known->second, true);
}

extern "C" int lbm_export_state(lbm_ctx* c, void* f, int precision) {
    if (!c) return LBM_EINVAL;
    if (!f) return fail(c, LBM_EINVAL, "f is NULL");
    if (precision != LBM_FP64 && precision != LBM_FP32) return fail(c, LBM_EINVAL, "precision must be LBM_FP64 or LBM_FP32");
    if (!c->have_fields) return fail(c, LBM_EINVAL, "lbm_set_fields has not been called");
    CK(cudaSetDevice(c->d.device));
    const Batch B = batch(c);
    const int ns = c->d.n_species;
    const Batch* pb = c->pull ? &B : nullptr;
    if (precision == LBM_FP64)
        CK(c->d.precision == LBM_FP64 ? launch_export(ns, (const double*)c->f[c->cur], (double*)f, c->c64, pb, c->stream)
                                      : launch_export(ns, (const float*)c->f[c->cur], (double*)f, c->c32, pb, c->stream));
    else
        CK(c->d.precision == LBM_FP64 ? launch_export(ns, (const double*)c->f[c->cur], (float*)f, c->c64, pb, c->stream)
                                      : launch_export(ns, (const float*)c->f[c->cur], (float*)f, c->c32, pb, c->stream));
    c->launches += 1;
    return LBM_OK;
}

extern "C" int lbm_get_fields(lbm_ctx* c, double* rho, double* u, double* f, int where) {
    if (!c) return LBM_EINVAL;
    if (!c->have_fields) return fail(c, LBM_EINVAL, "lbm_set_fields has not been called");
    if (where != LBM_HOST && where != LBM_DEVICE) return fail(c, LBM_EINVAL, "where must be LBM_HOST or LBM_DEVICE");
    CK(cudaSetDevice(c->d.device));
    const Batch B = batch(c);
    const int ns = c->d.n_species;
    const long long n = (long long)c->d.nx * c->d.nz;
    const cudaMemcpyKind kind = where == LBM_HOST ? cudaMemcpyDeviceToHost : cudaMemcpyDeviceToDevice;
    if (rho || u) {
        CK(enqueue_pass(c, c->cur, M_FIELDS, false, false, false));
        if (rho) CK(cudaMemcpyAsync(rho, c->staging, (size_t)ns * n * sizeof(double), kind, c->stream));
        if (u) CK(cudaMemcpyAsync(u, c->staging + ns * n, (size_t)2 * n * sizeof(double), kind, c->stream));
    }
    if (f) {
        if (!c->fexport) CK(cudaMalloc(&c->fexport, (size_t)ns * 9 * n * sizeof(double)));
        if (c->d.precision == LBM_FP64)
            CK(launch_export<double>(ns, (const double*)c->f[c->cur], c->fexport, c->c64, c->pull ? &B : nullptr,
                                     c->stream));
        else
            CK(launch_export<float>(ns, (const float*)c->f[c->cur], c->fexport, c->c32, c->pull ? &B : nullptr,
                                    c->stream));
        c->launches += 1;
        CK(cudaMemcpyAsync(f, c->fexport, (size_t)ns * 9 * n * sizeof(double), kind, c->stream));
    }
    CK(cudaStreamSynchronize(c->stream));
    return LBM_OK;
}

// ---------------------------------------------------------------------------------------
// Observables
// ---------------------------------------------------------------------------------------
// Entry i of the device observable buffers: a double (FP64 mode) or a (hi, lo) float pair
// (FP32 mode, compensated sums); widened here to FP64.
static double entry(const lbm_ctx* c, const double* buf, long long i) {
    if (c->d.precision == LBM_FP64) return buf[i];
    const float* p = reinterpret_cast<const float*>(buf) + 2 * i;
    return (double)p[0] + (double)p[1];
}

static void unpack(const lbm_ctx* c, const double* buf, lbm_obs* o, double scale) {
    const int nx = c->d.nx, nz = c->d.nz, ns = c->d.n_species;
    auto E = [&](long long i) { return entry(c, buf, i); };
    // the scalars: FP64 sums, in block order, of the reduction's block partials
    const long long ol = obs_len(nx, nz), nb = reduce_blocks(nx, nz);
    double sc[5] = {0.0, 0.0, 0.0, 0.0, 0.0};
    for (long long b = 0; b < nb; ++b)
        for (int k = 0; k < 5; ++k) sc[k] += E(ol + 5 * b + k);
    o->mass[0] = sc[0] * scale;
    o->mass[1] = ns == 2 ? sc[1] * scale : 0.0;
    o->momentum[0] = sc[2] * scale;
    o->momentum[1] = sc[3] * scale;
    o->gamma = sc[4] * scale;
    // wall forces: the sums of the wall profiles (of every lattice of a batch)
    const long long wb = O_PROF + 7LL * nz + 2LL * nx, wt = wb + nz;
    double fb = 0.0, ft = 0.0;
    if (c->d.z_boundary)
        for (int z = 0; z < nz; ++z) {
            fb += E(wb + z);
            ft += E(wt + z);
        }
    o->wall_force[0] = fb * scale;
    o->wall_force[1] = ft * scale;
    bool bad = E(O_BAD) != 0.0;
    for (int k = 0; k < 5; ++k) bad = bad || !std::isfinite(sc[k]);
    o->nonfinite = bad;
    o->step = c->step;
    const long long ux = O_PROF, rz = ux + nz, sx = rz + 2LL * nz, fl = sx + nz, ps = fl + nz, px = ps + nx;
    for (int z = 0; z < nz; ++z) {
        if (o->ux_z) o->ux_z[z] = E(ux + z) * scale;
        if (o->sxz_z) o->sxz_z[z] = E(sx + z) * scale;
        if (o->fluid_z) o->fluid_z[z] = E(fl + z) * scale;
        if (o->rho_z)
            for (int s = 0; s < ns; ++s) o->rho_z[s * nz + z] = E(rz + (long long)s * nz + z) * scale;
    }
    for (int x = 0; x < nx; ++x) {
        if (o->ps_x) o->ps_x[x] = E(ps + x) * scale;
        if (o->pxx_x) o->pxx_x[x] = E(px + x) * scale;
    }
}

// Lattice i of a batch from the row profiles of the observable buffer buf.
static void unpack_instance(const lbm_ctx* c, const double* buf, int i, lbm_obs* o, double scale) {
    const int nx = c->d.nx, nz = c->d.nz, ns = c->d.n_species;
    const InstGeom& g = c->inst[i];
    auto E = [&](long long k) { return entry(c, buf, k); };
    const long long ux = O_PROF, rz = ux + nz, sx = rz + 2LL * nz, fl = sx + nz, mx = fl + nz + 2LL * nx,
                    mz = mx + nz, wb = mz + nz, wt = wb + nz;
    double m[2] = {0.0, 0.0}, j[2] = {0.0, 0.0}, w[2] = {0.0, 0.0};
    for (int k = 0; k < g.nz; ++k) {
        const long long z = g.zrow0 + k;
        for (int s = 0; s < ns; ++s) m[s] += E(rz + (long long)s * nz + z);
        j[0] += E(mx + z);
        j[1] += E(mz + z);
        w[0] += E(wb + z);
        w[1] += E(wt + z);
        if (o->ux_z) o->ux_z[k] = E(ux + z) * scale;
        if (o->sxz_z) o->sxz_z[k] = E(sx + z) * scale;
        if (o->fluid_z) o->fluid_z[k] = E(fl + z) * scale;
        if (o->rho_z)
            for (int s = 0; s < ns; ++s) o->rho_z[s * g.nz + k] = E(rz + (long long)s * nz + z) * scale;
    }
    // the profiles are x-averages: sums over the lattice are nx times their sums over rows
    o->mass[0] = m[0] * nx * scale;
    o->mass[1] = m[1] * nx * scale;
    o->momentum[0] = j[0] * nx * scale;
    o->momentum[1] = j[1] * nx * scale;
    o->wall_force[0] = w[0] * scale;
    o->wall_force[1] = w[1] * scale;
    o->gamma = 0.0;
    o->nonfinite = E(O_BAD) != 0.0;
    o->step = c->step;
}

extern "C" int lbm_instance_observables(lbm_ctx* c, int i, lbm_obs* o, int averages) {
    if (!c) return LBM_EINVAL;
    if (!o) return fail(c, LBM_EINVAL, "out is NULL");
    if (i < 0 || i >= (int)c->inst.size()) return fail(c, LBM_EINVAL, "lattice %d not in the batch", i);
    if (!c->have_fields) return fail(c, LBM_EINVAL, "lbm_set_fields has not been called");
    CK(cudaSetDevice(c->d.device));
    if (averages) {
        CK(flush_pending(c));
        CK(cudaMemcpyAsync(c->host_out, c->avg, obs_bytes(c), cudaMemcpyDeviceToHost, c->stream));
        CK(cudaStreamSynchronize(c->stream));
        unpack_instance(c, c->host_out, i, o, c->samples > 0 ? 1.0 / (double)c->samples : 0.0);
        o->samples = c->samples;
        return LBM_OK;
    }
    CK(enqueue_pass(c, c->cur, M_OBS, true, false, false));
    CK(cudaMemcpyAsync(c->host_out, c->out, obs_bytes(c), cudaMemcpyDeviceToHost, c->stream));
    CK(cudaStreamSynchronize(c->stream));
    unpack_instance(c, c->host_out, i, o, 1.0);
    o->samples = 1;
    return o->nonfinite ? fail(c, LBM_ENONFINITE, "state holds a density <= 0, NaN or Inf") : LBM_OK;
}

extern "C" int lbm_observables(lbm_ctx* c, lbm_obs* o) {
    if (!c) return LBM_EINVAL;
    if (!o) return fail(c, LBM_EINVAL, "out is NULL");
    if (!c->have_fields) return fail(c, LBM_EINVAL, "lbm_set_fields has not been called");
    CK(cudaSetDevice(c->d.device));
    CK(enqueue_pass(c, c->cur, M_OBS, true, false, false));
    CK(cudaMemcpyAsync(c->host_out, c->out, obs_bytes(c), cudaMemcpyDeviceToHost, c->stream));
    CK(cudaStreamSynchronize(c->stream));
    unpack(c, c->host_out, o, 1.0);
    o->samples = 1;
    return o->nonfinite ? fail(c, LBM_ENONFINITE, "state holds a density <= 0, NaN or Inf") : LBM_OK;
}

extern "C" int lbm_averages(lbm_ctx* c, lbm_obs* o, int reset) {
    if (!c) return LBM_EINVAL;
    if (!o) return fail(c, LBM_EINVAL, "out is NULL");
    CK(cudaSetDevice(c->d.device));
    CK(flush_pending(c));
    CK(cudaMemcpyAsync(c->host_out, c->avg, obs_bytes(c), cudaMemcpyDeviceToHost, c->stream));
    CK(cudaStreamSynchronize(c->stream));
    const double n = (double)c->samples;
    unpack(c, c->host_out, o, n > 0 ? 1.0 / n : 0.0);
    o->samples = c->samples;
    if (reset) {
        CK(cudaMemsetAsync(c->avg, 0, obs_bytes(c), c->stream));
        c->samples = 0;
    }
    return LBM_OK;
}

// ---------------------------------------------------------------------------------------
// Asynchronous reads of the observables
// ---------------------------------------------------------------------------------------
// A record: the observable buffer as the reduction leaves it (obs_bytes), then a trailer.
struct ObsTrailer {
    double samples;  // states summed in the record (1: the current state)
    long long step;  // the step counter when the read was enqueued
    long long averages;
    long long pad_;
};

extern "C" long long lbm_observables_bytes(const lbm_ctx* c) {
    return c ? (long long)(obs_bytes(c) + sizeof(ObsTrailer)) : -1;
}

extern "C" int lbm_observables_enqueue(lbm_ctx* c, void* dst, int averages, int reset, long long* ticket) {
    if (!c) return LBM_EINVAL;
    if (!dst) return fail(c, LBM_EINVAL, "dst is NULL");
    if (!c->have_fields) return fail(c, LBM_EINVAL, "lbm_set_fields has not been called");
    CK(cudaSetDevice(c->d.device));
    // the trailer: written by the CPU into host memory, or on the device right after the buffer it
    // describes (then the two leave in one copy) -- a host-to-host cudaMemcpyAsync would make the
    // call wait for the stream
    static_assert(sizeof(ObsTrailer) == 32, "trailer layout");
    if (averages < 0 || averages > 2) return fail(c, LBM_EINVAL, "averages must be 0, 1 or 2");
    double* src;
    double samples;
    // a reduction left pending by the last observing step, to be added to the time sums by the
    // next step's launch
    const bool held = c->pull && c->pending && c->pending_acc;
    if (averages == 2 && held) {  // the sums as they stand: the pending sample goes to the next read
        src = c->avg;
        samples = (double)(c->samples - 1);
    } else if (averages) {
        CK(flush_pending(c));
        src = c->avg;
        samples = (double)c->samples;
    } else {
        CK(enqueue_pass(c, c->cur, M_OBS, true, false, false));
        src = c->out;
        samples = 1.0;
    }
    cudaPointerAttributes pa{};
    const bool host_dst = cudaPointerGetAttributes(&pa, dst) == cudaSuccess &&
                          (pa.type == cudaMemoryTypeHost || pa.type == cudaMemoryTypeUnregistered);
    cudaGetLastError();  // an unregistered pointer may leave an error behind
    if (host_dst) {
        // the trailer goes straight into host memory: the copy in flight writes other bytes
        ObsTrailer t{samples, c->step, averages ? 1 : 0, 0};
        memcpy(static_cast<char*>(dst) + obs_bytes(c), &t, sizeof t);
        CK(cudaMemcpyAsync(dst, src, obs_bytes(c), cudaMemcpyDefault, c->stream));
    } else {
        CK(launch_obs_trailer(reinterpret_cast<double*>(reinterpret_cast<char*>(src) + obs_bytes(c)), samples,
                              c->step, averages ? 1 : 0, c->stream));
        c->launches += 1;
        CK(cudaMemcpyAsync(dst, src, obs_bytes(c) + sizeof(ObsTrailer), cudaMemcpyDefault, c->stream));
    }
    if (averages && reset) {
        CK(cudaMemsetAsync(c->avg, 0, obs_bytes(c), c->stream));
        c->samples = averages == 2 && held ? 1 : 0;
    }
    cudaEvent_t& e = c->tev[c->tickets % 64];
    if (!e) CK(cudaEventCreateWithFlags(&e, cudaEventDisableTiming));
    CK(cudaEventRecord(e, c->stream));
    if (ticket) *ticket = c->tickets;
    c->tickets += 1;
    return LBM_OK;
}

// Where the device can write the host memory at p (pinned or registered): its device address,
// or null (pageable memory, device memory, unknown pointers).
static double* host_record_ptr(void* p) {
    cudaPointerAttributes pa{};
    const cudaError_t e = cudaPointerGetAttributes(&pa, p);
    cudaGetLastError();  // an unregistered pointer may leave an error behind
    if (e != cudaSuccess || pa.type != cudaMemoryTypeHost || !pa.devicePointer) return nullptr;
    return static_cast<double*>(pa.devicePointer);
}

extern "C" int lbm_step_read(lbm_ctx* c, int nsteps, void* dst, long long stride, int averages, int reset,
                             long long* ticket) {
    if (!c) return LBM_EINVAL;
    if (nsteps < 0) return fail(c, LBM_EINVAL, "nsteps < 0");
    if (!dst && nsteps > 0) return fail(c, LBM_EINVAL, "dst is NULL");
    if (stride < lbm_observables_bytes(c)) return fail(c, LBM_EINVAL, "stride is below lbm_observables_bytes");
    if (!c->have_fields) return fail(c, LBM_EINVAL, "lbm_set_fields has not been called");
    CK(cudaSetDevice(c->d.device));
    // Every step samples and every record holds the one completed sample (averages = 2 with
    // reset): each launch's folded reduction writes the sample it completes straight into that
    // step's record in pinned host memory, so no copy or reset runs between two step kernels.
    // The time sums stay cleared and keep only the sample still pending, as the plain path
    // leaves them.  The first step takes the plain path when the sums hold more than that.
    double* const dev_dst = (c->pull && averages == 2 && reset && c->observe_every == 1 && !c->profiling)
                                ? host_record_ptr(dst) : nullptr;
    const size_t ob = (size_t)obs_bytes(c);
    for (int i = 0; i < nsteps; ++i) {
        char* const rec = static_cast<char*>(dst) + (long long)i * stride;
        const bool held = c->pending && c->pending_acc;
        if (dev_dst && (c->samples == (held ? 1 : 0))) {
            if (!held) memset(rec, 0, ob);  // no sample completes in this launch
            const ObsTrailer t{held ? 1.0 : 0.0, c->step + 1, 1, 0};
            memcpy(rec + ob, &t, sizeof t);
            c->rec_dst = reinterpret_cast<double*>(reinterpret_cast<char*>(dev_dst) + (long long)i * stride);
            const cudaError_t e = enqueue_pass(c, c->cur, M_WRITE | M_OBS, true, true, true);
            c->rec_dst = nullptr;
            CK(e);
            c->samples = 1;  // the sample of this step, pending; the one before went into the record
            c->cur ^= 1;
            c->step += 1;
            continue;
        }
        const int rc = lbm_step(c, 1);
        if (rc != LBM_OK) return rc;
        const int rr = lbm_observables_enqueue(c, rec, averages, reset, ticket);
        if (rr != LBM_OK) return rr;
    }
    if (dev_dst && nsteps > 0) {  // one event for the run: its last record
        cudaEvent_t& e = c->tev[c->tickets % 64];
        if (!e) CK(cudaEventCreateWithFlags(&e, cudaEventDisableTiming));
        CK(cudaEventRecord(e, c->stream));
        if (ticket) *ticket = c->tickets;
        c->tickets += 1;
    }
    return LBM_OK;
}

extern "C" int lbm_wait(lbm_ctx* c, long long ticket) {
    if (!c) return LBM_EINVAL;
    if (ticket < 0 || ticket >= c->tickets) return fail(c, LBM_EINVAL, "ticket %lld was not issued", ticket);
    CK(cudaSetDevice(c->d.device));
    if (ticket < c->tickets - 64)
        CK(cudaStreamSynchronize(c->stream));  // its event was reused: wait for everything
    else
        CK(cudaEventSynchronize(c->tev[ticket % 64]));
    return LBM_OK;
}

extern "C" int lbm_observables_unpack(const lbm_ctx* c, const void* src, lbm_obs* o) {
    if (!c || !src || !o) return LBM_EINVAL;
    const double* buf = static_cast<const double*>(src);
    ObsTrailer t;
    memcpy(&t, static_cast<const char*>(src) + obs_bytes(c), sizeof t);
    unpack(c, buf, o, t.samples > 0 ? 1.0 / t.samples : 0.0);
    o->step = t.step;
    o->samples = (long long)t.samples;
    return o->nonfinite && !t.averages ? LBM_ENONFINITE : LBM_OK;
}

extern "C" int lbm_synchronize(lbm_ctx* c) {
    if (!c) return LBM_EINVAL;
    CK(cudaSetDevice(c->d.device));
    CK(cudaStreamSynchronize(c->stream));
    int flag = 0;
    CK(cudaMemcpy(&flag, c->flag, sizeof(int), cudaMemcpyDeviceToHost));
    if (flag & 4)
        return fail(c, LBM_EINVAL, "a snapshot restored by lbm_restore_own had been overwritten since this "
                                   "context wrote it: the restored state is not valid");
    if (flag & 2) return fail(c, LBM_ETIMEOUT, "a bounded device-side wait for a tile load gave up");
    if (flag & 1) return fail(c, LBM_ENONFINITE, "a step met a density <= 0, NaN or Inf");
    return LBM_OK;
}

extern "C" long long lbm_launch_count(const lbm_ctx* c) { return c ? c->launches : -1; }

extern "C" int lbm_profile(lbm_ctx* c, int enable) {
    if (!c) return LBM_EINVAL;
    CK(cudaSetDevice(c->d.device));
    CK(cudaStreamSynchronize(c->stream));
    c->profiling = enable != 0;
    c->ev_used = 0;
    c->aev_used = 0;
    return LBM_OK;
}

extern "C" int lbm_profile_read_adjoint(lbm_ctx* c, double* ms, long long* steps) {
    if (!c) return LBM_EINVAL;
    CK(cudaSetDevice(c->d.device));
    CK(cudaStreamSynchronize(c->stream));
    double total[3] = {0.0, 0.0, 0.0};
    for (size_t k = 0; k + 5 < c->aev_used; k += 6)
        for (int j = 0; j < 3; ++j) {
            float t = 0.f;
            CK(cudaEventElapsedTime(&t, c->aev[k + 2 * j], c->aev[k + 2 * j + 1]));
            total[j] += t;
        }
    if (ms)
        for (int j = 0; j < 3; ++j) ms[j] = total[j];
    if (steps) *steps = (long long)(c->aev_used / 6);
    return LBM_OK;
}

extern "C" int lbm_profile_read(lbm_ctx* c, double* ms, long long* n) {
    if (!c) return LBM_EINVAL;
    CK(cudaSetDevice(c->d.device));
    CK(cudaStreamSynchronize(c->stream));
    double total = 0.0;
    for (size_t k = 0; k + 1 < c->ev_used; k += 2) {
        float t = 0.f;
        CK(cudaEventElapsedTime(&t, c->ev[k], c->ev[k + 1]));
        total += t;
    }
    if (ms) *ms = total;
    if (n) *n = (long long)(c->ev_used / 2);
    return LBM_OK;
}

extern "C" const char* lbm_last_error(const lbm_ctx* c) { return c ? c->err.c_str() : g_create_error.c_str(); }

extern "C" int lbm_abi_version(void) { return LBM_ABI_VERSION; }

extern "C" int lbm_selftest_wait(lbm_ctx* c, long long cycles) {
    if (!c) return LBM_EINVAL;
    if (cycles < 1 || cycles > 4000000000LL) return fail(c, LBM_EINVAL, "cycles out of range");
    CK(cudaSetDevice(c->d.device));
    int saved = 0;
    CK(cudaMemcpyAsync(&saved, c->flag, sizeof(int), cudaMemcpyDeviceToHost, c->stream));
    CK(cudaStreamSynchronize(c->stream));
    CK(launch_wait_selftest(c->flag, cycles, c->stream));
    c->launches += 1;
    int flag = 0;
    CK(cudaMemcpyAsync(&flag, c->flag, sizeof(int), cudaMemcpyDeviceToHost, c->stream));
    CK(cudaStreamSynchronize(c->stream));
    CK(cudaMemcpyAsync(c->flag, &saved, sizeof(int), cudaMemcpyHostToDevice, c->stream));
    CK(cudaStreamSynchronize(c->stream));
    if (flag & 2) return fail(c, LBM_ETIMEOUT, "the self-test wait expired after %lld cycles (expected)", cycles);
    return LBM_OK;
}

// Autotuner of the pull kernel's launch shapes: every candidate (pipeline depth, tile width) steps
// the context's own lattices `steps` times with the current sampling, timed by events; the
// fastest is kept for the kind of pass tuned (with or without observables).  The state, the time
// sums and the step count are put back afterwards, so tuning does not advance the simulation.
// ms[i]: milliseconds per step of candidate i, 0 for a shape the context does not have.
static int autotune_shapes(lbm_ctx* c, int steps, const int (*cand)[2], int ncand, int* pick, double* ms) {
    if (steps < 1 || steps > 10000) return fail(c, LBM_EINVAL, "steps must be in [1, 10000]");
    if (!c->have_fields) return fail(c, LBM_EINVAL, "lbm_set_fields has not been called");
    CK(cudaSetDevice(c->d.device));
    CK(flush_pending(c));
    const size_t fbytes = (size_t)c->d.n_species * 9 * c->plane * c->esize;
    void* save = nullptr;
    CK(cudaMalloc(&save, 2 * fbytes + obs_bytes(c) + sizeof(int)));
    unsigned char* sv = static_cast<unsigned char*>(save);
    cudaError_t e = cudaMemcpyAsync(sv, c->f[0], fbytes, cudaMemcpyDeviceToDevice, c->stream);
    if (e == cudaSuccess) e = cudaMemcpyAsync(sv + fbytes, c->f[1], fbytes, cudaMemcpyDeviceToDevice, c->stream);
    if (e == cudaSuccess) e = cudaMemcpyAsync(sv + 2 * fbytes, c->avg, obs_bytes(c), cudaMemcpyDeviceToDevice, c->stream);
    if (e == cudaSuccess)
        e = cudaMemcpyAsync(sv + 2 * fbytes + obs_bytes(c), c->flag, sizeof(int), cudaMemcpyDeviceToDevice, c->stream);
    const int cls = c->observe_every > 0 ? 1 : 0;  // the pass kind tuned: with or without observables
    const bool ob = c->observe_every > 0;
    const int cur = c->cur, saved_stages = c->stages[cls], saved_width = c->width[cls];
    const long long step = c->step, samples = c->samples, launches = c->launches;
    const bool prof = c->profiling;
    c->profiling = false;
    double best = 1e300;
    int best_i = -1;
    cudaEvent_t a = nullptr, b = nullptr;
    if (e == cudaSuccess) e = cudaEventCreate(&a);
    if (e == cudaSuccess) e = cudaEventCreate(&b);
    const int pm = M_WRITE | (ob ? M_OBS | (c->d.z_boundary == LBM_PERIODIC ? M_PERIODIC : 0) : 0);
    for (int i = 0; i < ncand && e == cudaSuccess; ++i) {
        ms[i] = 0.0;
        const int st = cand[i][0], w = cand[i][1];
        if (w == 64 && c->pull_grid[pm][st - 1][1] < 1) continue;  // not built for this context
        c->stages[cls] = st;
        c->width[cls] = w;
        for (int k = 0; k < 2 + steps && e == cudaSuccess; ++k) {  // two warm-up steps, then the timed ones
            if (k == 2) e = cudaEventRecord(a, c->stream);
            if (e == cudaSuccess) e = enqueue_pass(c, c->cur, M_WRITE | (ob ? M_OBS : 0), ob, ob, true);
            c->cur ^= 1;
        }
        if (e == cudaSuccess) e = cudaEventRecord(b, c->stream);
        if (e == cudaSuccess) e = cudaEventSynchronize(b);
        float t = 0.f;
        if (e == cudaSuccess) e = cudaEventElapsedTime(&t, a, b);
        ms[i] = (double)t / steps;
        if (e == cudaSuccess && ms[i] < best) {
            best = ms[i];
            best_i = i;
        }
    }
    // put the state back
    c->pending = false;
    c->cur = cur;
    if (e == cudaSuccess) e = cudaMemcpyAsync(c->f[0], sv, fbytes, cudaMemcpyDeviceToDevice, c->stream);
    if (e == cudaSuccess) e = cudaMemcpyAsync(c->f[1], sv + fbytes, fbytes, cudaMemcpyDeviceToDevice, c->stream);
    if (e == cudaSuccess) e = cudaMemcpyAsync(c->avg, sv + 2 * fbytes, obs_bytes(c), cudaMemcpyDeviceToDevice, c->stream);
    if (e == cudaSuccess)
        e = cudaMemcpyAsync(c->flag, sv + 2 * fbytes + obs_bytes(c), sizeof(int), cudaMemcpyDeviceToDevice, c->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(c->stream);
    if (a) cudaEventDestroy(a);
    if (b) cudaEventDestroy(b);
    cudaFree(save);
    c->step = step;
    c->samples = samples;
    c->launches = launches;
    c->profiling = prof;
    const bool ok = e == cudaSuccess && best_i >= 0;
    c->stages[cls] = ok ? cand[best_i][0] : saved_stages;
    c->width[cls] = ok ? cand[best_i][1] : saved_width;
    drop_graphs(c);
    CK(e);
    *pick = best_i;
    return LBM_OK;
}

extern "C" int lbm_autotune(lbm_ctx* c, int steps, int* chosen, double* ms_per_step) {
    if (!c) return LBM_EINVAL;
    if (steps < 1 || steps > 10000) return fail(c, LBM_EINVAL, "steps must be in [1, 10000]");
    if (!c->have_fields) return fail(c, LBM_EINVAL, "lbm_set_fields has not been called");
    if (!c->pull) {  // nothing to choose for the other kernels
        if (chosen) *chosen = 0;
        return LBM_OK;
    }
    const int w = c->width[c->observe_every > 0 ? 1 : 0];
    const int cand[2][2] = {{1, w}, {2, w}};
    double ms[2] = {0.0, 0.0};
    int pick = -1;
    const int rc = autotune_shapes(c, steps, cand, 2, &pick, ms);
    if (rc != LBM_OK) return rc;
    if (chosen) *chosen = cand[pick][0];
    if (ms_per_step) {
        ms_per_step[0] = ms[0];
        ms_per_step[1] = ms[1];
    }
    return LBM_OK;
}

extern "C" int lbm_autotune_tiles(lbm_ctx* c, int steps, int* width, int* depth, double* ms_per_step) {
    if (!c) return LBM_EINVAL;
    if (!c->pull) return fail(c, LBM_EINVAL, "tile shapes are the PULL kernel's");
    const int cand[4][2] = {{1, 32}, {2, 32}, {1, 64}, {2, 64}};
    double ms[4] = {0.0, 0.0, 0.0, 0.0};
    int pick = -1;
    const int rc = autotune_shapes(c, steps, cand, 4, &pick, ms);
    if (rc != LBM_OK) return rc;
    if (depth) *depth = cand[pick][0];
    if (width) *width = cand[pick][1];
    if (ms_per_step)
        for (int i = 0; i < 4; ++i) ms_per_step[i] = ms[i];
    return LBM_OK;
}

extern "C" int lbm_set_tile_shape(lbm_ctx* c, int width, int depth) {
    if (!c) return LBM_EINVAL;
    if (!c->pull) return fail(c, LBM_EINVAL, "tile shapes are the PULL kernel's");
    if ((width != 32 && width != 64) || (depth != 1 && depth != 2))
        return fail(c, LBM_EINVAL, "width must be 32 or 64 and depth 1 or 2");
    if (width == 64 && c->d.precision != LBM_FP32) return fail(c, LBM_EINVAL, "width 64 is built for FP32 only");
    CK(cudaSetDevice(c->d.device));
    for (int k = 0; k < 2; ++k) {
        c->stages[k] = depth;
        c->width[k] = width;
    }
    drop_graphs(c);
    return LBM_OK;
}

// ---------------------------------------------------------------------------------------
// Discrete adjoint (periodic single lattice)
// ---------------------------------------------------------------------------------------
static int adjoint_ready(lbm_ctx* c, AdjConst& A, int precision) {
    if (precision != LBM_FP64 && precision != LBM_FP32) return fail(c, LBM_EINVAL, "precision must be LBM_FP64 or LBM_FP32");
    if (c->d.z_boundary != LBM_PERIODIC) return fail(c, LBM_EINVAL, "the adjoint needs a periodic lattice");
    if (c->inst.size() > 1) return fail(c, LBM_EINVAL, "the adjoint is for a single lattice, not a batch");
    CK(cudaSetDevice(c->d.device));
    if (!c->adj_scratch) CK(cudaMalloc(&c->adj_scratch, adjoint_scratch_bytes(c->d.nx, c->d.nz, c->d.n_species)));
    fill_adj_const(A, c->p, c->d.nx, c->d.nz, c->d.n_species, c->inst.empty() ? c->p.body_force : c->inst[0].g);
    return LBM_OK;
}

static size_t state_values(const lbm_ctx* c) { return (size_t)c->d.n_species * 9 * c->d.nx * c->d.nz; }

extern "C" int lbm_record_states(lbm_ctx* c, int nsteps, void* states, int precision) {
    if (!c) return LBM_EINVAL;
    if (nsteps < 0 || (nsteps > 0 && !states)) return fail(c, LBM_EINVAL, "nsteps < 0 or states is NULL");
    if (precision != LBM_FP64 && precision != LBM_FP32) return fail(c, LBM_EINVAL, "precision must be LBM_FP64 or LBM_FP32");
    if (!c->have_fields) return fail(c, LBM_EINVAL, "lbm_set_fields has not been called");
    CK(cudaSetDevice(c->d.device));
    const size_t bytes = state_values(c) * (precision == LBM_FP32 ? sizeof(float) : sizeof(double));
    // the pull kernel writes the state it reads (M_RECORD) when the record is in its own precision,
    // the lattice is one lattice, and the step does not sample; otherwise export, then step
    const bool fused = c->pull && c->inst.size() == 1 && precision == c->d.precision;
    for (int k = 0; k < nsteps; ++k) {
        void* dst = static_cast<char*>(states) + k * bytes;
        if (fused && !observe_now(c, c->step)) {
            c->rec = dst;
            const cudaError_t e = enqueue_pass(c, c->cur, M_WRITE | M_RECORD, false, false, true);
            c->rec = nullptr;
            CK(e);
            c->cur ^= 1;
            c->step += 1;
        } else {
            if (int r = lbm_export_state(c, dst, precision)) return r;
            if (int r = lbm_step(c, 1)) return r;
        }
    }
    return LBM_OK;
}

template <typename T>
static int adjoint_steps(lbm_ctx* c, const AdjConst& A, int nsteps, const T* states, const T* lam_in, T* lam_a,
                         T* lam_b, T* lam_user, double* grad) {
    const T* out = nullptr;
    cudaEvent_t* ev = nullptr;
    if (c->profiling && nsteps > 0) {
        while (c->aev.size() < c->aev_used + 6 * (size_t)nsteps) {
            cudaEvent_t e;
            CK(cudaEventCreate(&e));
            c->aev.push_back(e);
        }
        ev = c->aev.data() + c->aev_used;
        c->aev_used += 6 * (size_t)nsteps;
    }
    CK(launch_adjoint_steps<T>(A, nsteps, states, (long long)state_values(c), lam_in, lam_a, lam_b, &out, grad,
                               c->adj_scratch, ev, c->stream));
    if (out != lam_user)
        CK(cudaMemcpyAsync(lam_user, out, state_values(c) * sizeof(T), cudaMemcpyDeviceToDevice, c->stream));
    c->launches += 2LL * nsteps + (nsteps > 0 ? 2 : 0);
    return LBM_OK;
}

extern "C" int lbm_adjoint_step(lbm_ctx* c, const void* f, const void* lam_next, void* lam, double* grad,
                                int precision) {
    if (!c) return LBM_EINVAL;
    if (!f || !lam_next || !lam || !grad) return fail(c, LBM_EINVAL, "NULL pointer");
    if (lam == lam_next || lam == f) return fail(c, LBM_EINVAL, "lam must not overlap lam_next or f");
    AdjConst A;
    if (int r = adjoint_ready(c, A, precision)) return r;
    if (precision == LBM_FP64)
        return adjoint_steps<double>(c, A, 1, (const double*)f, (const double*)lam_next, (double*)lam, nullptr,
                                     (double*)lam, grad);
    return adjoint_steps<float>(c, A, 1, (const float*)f, (const float*)lam_next, (float*)lam, nullptr, (float*)lam,
                                grad);
}

extern "C" int lbm_adjoint_steps(lbm_ctx* c, int nsteps, const void* states, void* lam, double* grad, int precision) {
    if (!c) return LBM_EINVAL;
    if (nsteps < 0 || !lam || !grad || (nsteps > 0 && !states)) return fail(c, LBM_EINVAL, "bad argument");
    AdjConst A;
    if (int r = adjoint_ready(c, A, precision)) return r;
    if (!c->adj_lam) CK(cudaMalloc(&c->adj_lam, state_values(c) * sizeof(double)));
    // the first step writes the context's buffer, the second the caller's (read no more), ...
    if (precision == LBM_FP64)
        return adjoint_steps<double>(c, A, nsteps, (const double*)states, (const double*)lam, (double*)c->adj_lam,
                                     (double*)lam, (double*)lam, grad);
    return adjoint_steps<float>(c, A, nsteps, (const float*)states, (const float*)lam, (float*)c->adj_lam,
                                (float*)lam, (float*)lam, grad);
}

extern "C" int lbm_adjoint_objective(lbm_ctx* c, const void* f, const double* target_u, const double* target_rho,
                                     double* J, void* dJdf, int precision) {
    if (!c) return LBM_EINVAL;
    if (!f || !target_u || !target_rho || !J) return fail(c, LBM_EINVAL, "NULL pointer");
    AdjConst A;
    if (int r = adjoint_ready(c, A, precision)) return r;
    if (precision == LBM_FP64)
        CK(launch_adjoint_objective<double>(A, (const double*)f, target_u, target_rho, J, (double*)dJdf,
                                            c->adj_scratch, c->stream));
    else
        CK(launch_adjoint_objective<float>(A, (const float*)f, target_u, target_rho, J, (float*)dJdf, c->adj_scratch,
                                           c->stream));
    c->launches += dJdf ? 3 : 2;
    return LBM_OK;
}

extern "C" int lbm_adjoint_initial(lbm_ctx* c, const void* lam0, double* g_rho, int precision) {
    if (!c) return LBM_EINVAL;
    if (!lam0 || !g_rho) return fail(c, LBM_EINVAL, "NULL pointer");
    AdjConst A;
    if (int r = adjoint_ready(c, A, precision)) return r;
    if (precision == LBM_FP64)
        CK(launch_adjoint_initial<double>(A, (const double*)lam0, g_rho, c->stream));
    else
        CK(launch_adjoint_initial<float>(A, (const float*)lam0, g_rho, c->stream));
    c->launches += 1;
    return LBM_OK;
}
