// C ABI of the super-droplet library: context life cycle, argument checks,
// field marshalling, the order of launches in step_sync / step_async
// (paper Sec. 5.2.1-5.2.2) and the diagnostics.  Every numerical step runs
// in the kernels of this directory; host code only moves arguments.
#include <math.h>
#include <stdio.h>
#include <stdlib.h>
#include <string.h>

#include <chrono>
#include <thread>

#include <nvtx3/nvToolsExt.h>

#include "sdm_internal.cuh"

using namespace sdm;

namespace {

thread_local std::string g_init_err;

sdm_status fail(sdm_ctx *c, sdm_status s, const std::string &msg) {
    if (c) c->err = msg;
    else g_init_err = msg;
    return s;
}

sdm_status cuda_fail(sdm_ctx *c, cudaError_t e, const char *where) {
    return fail(c, SDM_ECUDA, std::string(where) + ": " + cudaGetErrorString(e));
}

#define CK(call, where)                                 \
    do {                                                \
        cudaError_t e_ = (call);                        \
        if (e_ != cudaSuccess) return cuda_fail(c, e_, where); \
    } while (0)

int nd_present(const sdm_ctx *c) {
    return (c->grid.nx > 0) + (c->grid.ny > 0) + (c->grid.nz > 0);
}

// shape of a cell-centred field, or of an edge field along dimension `edge`
// (0 x, 1 y, 2 z; -1 centred), without absent dimensions
int field_shape(const sdm_ctx *c, int edge, int *shape) {
    const int n[3] = {c->grid.nx, c->grid.ny, c->grid.nz};
    int d = 0;
    for (int a = 0; a < 3; ++a)
        if (n[a] > 0) shape[d++] = n[a] + (a == edge ? 1 : 0);
    if (d == 0) shape[d++] = 1;
    return d;
}

// copy a caller field described by sdm_arr into a contiguous device array
sdm_status field_in(sdm_ctx *c, double *dev, const sdm_arr &a, int edge, const char *name) {
    int shape[3];
    const int nd = field_shape(c, edge, shape);
    int64_t total = 1;
    for (int d = 0; d < nd; ++d) total *= shape[d];
    if (nd_present(c) == 0 || !a.strides) {  // box: one value, or a contiguous array
        if (a.on_device) CK(cudaMemcpyAsync(dev, a.data_zero, total * 8, cudaMemcpyDeviceToDevice, c->stream), name);
        else CK(cudaMemcpyAsync(dev, a.data_zero, total * 8, cudaMemcpyHostToDevice, c->stream), name);
        return SDM_OK;
    }
    if (a.on_device) {
        CK(launch_field_gather(dev, a.data_zero, a.strides, nd, shape, c->stream), name);
        c->tacc.launches += 1;
        return SDM_OK;
    }
    if (a.strides[nd - 1] != 1)
        return fail(c, SDM_ENOTSUP, std::string(name) + ": host arrays need unit innermost stride");
    const int64_t inner = shape[nd - 1];
    const int64_t rows = total / inner;
    // rows of the innermost dimension, each at its strided host address
    const int64_t outer = nd == 3 ? shape[0] : 1;
    const int64_t mid = nd >= 2 ? shape[nd - 2] : 1;
    for (int64_t i = 0; i < outer; ++i) {
        const double *src = a.data_zero + (nd == 3 ? i * a.strides[0] : 0);
        const int64_t pitch = nd >= 2 ? a.strides[nd - 2] : inner;
        CK(cudaMemcpy2DAsync(dev + i * mid * inner, inner * 8, src, pitch * 8, inner * 8, mid,
                             cudaMemcpyHostToDevice, c->stream), name);
    }
    (void)rows;
    return SDM_OK;
}

sdm_status field_out(sdm_ctx *c, const sdm_arr &a, const double *dev, const char *name) {
    int shape[3];
    const int nd = field_shape(c, -1, shape);
    int64_t total = 1;
    for (int d = 0; d < nd; ++d) total *= shape[d];
    if (nd_present(c) == 0 || !a.strides) {
        CK(cudaMemcpyAsync(a.data_zero, dev, total * 8,
                           a.on_device ? cudaMemcpyDeviceToDevice : cudaMemcpyDeviceToHost, c->stream), name);
        return SDM_OK;
    }
    if (a.on_device) {
        CK(launch_field_scatter(a.data_zero, dev, a.strides, nd, shape, c->stream), name);
        c->tacc.launches += 1;
        return SDM_OK;
    }
    if (a.strides[nd - 1] != 1)
        return fail(c, SDM_ENOTSUP, std::string(name) + ": host arrays need unit innermost stride");
    const int64_t inner = shape[nd - 1];
    const int64_t outer = nd == 3 ? shape[0] : 1;
    const int64_t mid = nd >= 2 ? shape[nd - 2] : 1;
    for (int64_t i = 0; i < outer; ++i) {
        double *dst = a.data_zero + (nd == 3 ? i * a.strides[0] : 0);
        const int64_t pitch = nd >= 2 ? a.strides[nd - 2] : inner;
        CK(cudaMemcpy2DAsync(dst, pitch * 8, dev + i * mid * inner, inner * 8, inner * 8, mid,
                             cudaMemcpyDeviceToHost, c->stream), name);
    }
    return SDM_OK;
}

// ---- initial dry-radius range (the same reading as the test oracle):
// super-droplets uniform in ln r over [lo, hi] each stand for a slice
// (hi - lo)/sd_conc of ln r; the range is narrowed to the outermost radii
// where n(ln r) dlnr dV >= 1, starting from [1 nm, 10 um], 8 passes.
double n_lnr_host(const std::vector<sdm_lognormal> &modes, double kap, double lnr) {
    double s = 0.0;
    for (const auto &m : modes) {
        if (m.kappa != kap) continue;
        const double ls = log(m.sigma);
        const double q = (lnr - log(m.rm)) / ls;
        s += m.n_stp / (sqrt(2.0 * phys::pi) * ls) * exp(-0.5 * q * q);
    }
    return s;
}

bool rd_range(const sdm_ctx *c, double kap, double *lo_out, double *hi_out) {
    return sdm::rd_range_modes(c->modes, kap, c->oi.sd_conc, c->oi.dx * c->oi.dy * c->oi.dz, lo_out,
                               hi_out);
}

}  // namespace

bool sdm::rd_range_modes(const std::vector<sdm_lognormal> &modes, double kap, int64_t sd_conc, double dV,
                         double *lo_out, double *hi_out) {
    const double L0 = log(1e-9), L1 = log(1e-5);
    const int NG = 1000;
    double lo = L0, hi = L1;
    for (int pass = 0; pass < 8; ++pass) {
        const double dlnr = (hi - lo) / sd_conc;
        auto w = [&](double l) { return n_lnr_host(modes, kap, l) * dlnr * dV; };
        int jlo = -1, jhi = -1;
        for (int j = 0; j <= NG; ++j)
            if (w(L0 + (L1 - L0) * j / NG) >= 1.0) {
                jlo = j;
                break;
            }
        for (int j = NG; j >= 0; --j)
            if (w(L0 + (L1 - L0) * j / NG) >= 1.0) {
                jhi = j;
                break;
            }
        if (jlo < 0 || jhi < 0) return false;
        double nlo = L0 + (L1 - L0) * jlo / NG, nhi = L0 + (L1 - L0) * jhi / NG;
        if (jlo > 0) {
            double b0 = L0 + (L1 - L0) * (jlo - 1) / NG, b1 = nlo;
            for (int it = 0; it < 100; ++it) {
                const double m = 0.5 * (b0 + b1);
                if (w(m) >= 1.0) b1 = m;
                else b0 = m;
            }
            nlo = b1;
        }
        if (jhi < NG) {
            double b0 = nhi, b1 = L0 + (L1 - L0) * (jhi + 1) / NG;
            for (int it = 0; it < 100; ++it) {
                const double m = 0.5 * (b0 + b1);
                if (w(m) >= 1.0) b0 = m;
                else b1 = m;
            }
            nhi = b0;
        }
        lo = nlo;
        hi = nhi;
    }
    *lo_out = lo;
    *hi_out = hi;
    return true;
}

namespace {

// Fault injection on the host, for tests of the allocation-failure path
// without a GPU fault: with SDM_FAIL_ALLOC=k in the environment, the k-th
// device allocation of each sdm_init reports cudaErrorMemoryAllocation
// instead of allocating (sdm_init then returns SDM_ENOMEM and frees what it
// had).  Read at every sdm_init; unset, it costs one getenv per init.
static thread_local int g_fail_alloc = 0;

template <class T>
cudaError_t dalloc(T **p, size_t n) {
    *p = nullptr;
    if (n == 0) return cudaSuccess;
    if (g_fail_alloc > 0 && --g_fail_alloc == 0) return cudaErrorMemoryAllocation;  // injected
    return cudaMalloc((void **)p, n * sizeof(T));
}

void free_ctx(sdm_ctx *c) {
    if (!c) return;
    for (int b = 0; b < 2; ++b) {
        SdArrays &s = c->buf[b];
        cudaFree(s.N);
        cudaFree(s.rw2);
        cudaFree(s.rd3);
        cudaFree(s.kappa);
        cudaFree(s.x);
        cudaFree(s.y);
        cudaFree(s.z);
        cudaFree(s.uid);
    }
    cudaFree(c->newcell);
    cudaFree(c->slot);
    cudaFree(c->perm);
    cudaFree(c->count);
    cudaFree(c->xch_flag);
    cudaFree(c->xch_off);
    cudaFree(c->xch_tmp);
    cudaFree(c->offset);
    cudaFree(c->bigcells);
    cudaFree(c->huge);
    cudaFree(c->th);
    cudaFree(c->rv);
    cudaFree(c->rhod);
    cudaFree(c->amb);
    cudaFree(c->outbuf);
    cudaFree(c->spec_buf);
    cudaFree(c->spec_edges);
    cudaFree(c->cs_rec[0]);
    cudaFree(c->cs_rec[1]);
    cudaFree(c->cs_cell);
    cudaFree(c->cs_x1);
    cudaFree(c->cs_cnt);
    cudaFree(c->cond_order);
    cudaFree(c->cond_cost);
    cudaFree(c->euler_tmp);
    cudaFree(c->euler_prof);
    for (int d = 0; d < 3; ++d) cudaFree(c->cedge[d]);
    for (int d = 0; d < 3; ++d) cudaFree(c->rhoC[d]);
    cudaFree(c->scan_tmp);
    cudaFree(c->rc_tmp);
    cudaFree(c->rc_sel);
    cudaFree(c->dstats);
    if (c->hstats) cudaFreeHost(c->hstats);
    for (auto &t : c->timers) {
        cudaEventDestroy(t.a);
        cudaEventDestroy(t.b);
    }
    for (auto e : c->event_pool) cudaEventDestroy(e);
    if (c->done_event) cudaEventDestroy(c->done_event);
    if (c->own_stream && c->stream) cudaStreamDestroy(c->stream);
    delete c;
}

enum { PH_COND, PH_RECYCLE, PH_MOVE, PH_SORT, PH_COAL, PH_DIAG, PH_COPY, PH_EULER };
// NVTX range names of the phases (a profiler's timeline shows them; without
// one attached the calls cost next to nothing)
static const char *const kPhaseName[] = {"sdm condensation", "sdm recycling", "sdm transport",  "sdm sort",
                                         "sdm coalescence",  "sdm diagnostics", "sdm field copies", "sdm eulerian"};

cudaEvent_t pool_event(sdm_ctx *c) {
    if (!c->event_pool.empty()) {
        cudaEvent_t e = c->event_pool.back();
        c->event_pool.pop_back();
        return e;
    }
    cudaEvent_t e = nullptr;
    cudaEventCreate(&e);
    return e;
}

struct Phase {  // records a CUDA-event pair around a group of launches
    sdm_ctx *c;
    int ph;
    cudaEvent_t a = nullptr;
    Phase(sdm_ctx *c_, int ph_) : c(c_), ph(ph_) {
        nvtxRangePushA(kPhaseName[ph_]);
        if (c->timing) {
            a = pool_event(c);
            cudaEventRecord(a, c->stream);
        }
    }
    ~Phase() {
        nvtxRangePop();
        if (c->timing && a) {
            cudaEvent_t b = pool_event(c);
            cudaEventRecord(b, c->stream);
            c->timers.push_back(PhaseTimer{a, b, ph});
        }
    }
};

sdm_status check_flags(sdm_ctx *c, unsigned flags) {
    if (flags & kFlagNumeric)
        return fail(c, SDM_ENUMERIC, "a kernel produced a non-finite radius or field value");
    if (flags & kFlagBigCell)
        return fail(c, SDM_ENOTSUP, "a grid cell holds more than 8192 super-droplets and the context has no "
                                    "scratch for such cells (its initial cells hold at most 8192)");
    return SDM_OK;
}

sdm_status pull_stats(sdm_ctx *c) {
    CK(cudaMemcpyAsync(c->hstats, c->dstats, sizeof(DevStats), cudaMemcpyDeviceToHost, c->stream),
       "stats copy");
    CK(cudaStreamSynchronize(c->stream), "stats sync");
    c->mirror = *c->hstats;
    return SDM_OK;
}

// regroup after positions changed outside a step: cells from positions,
// counting sort, gather without coalescence
sdm_status regroup(sdm_ctx *c) {
    sdm_opts o{0, 0, 0, 0, 44.0, 1, 1};
    CK(launch_ambient(c), "ambient");
    CK(launch_move(c, o), "move");
    CK(launch_regroup(c), "scan");
    CK(launch_coalesce(c, o, false), "gather");
    c->cur ^= 1;
    c->layout_dirty = false;
    return SDM_OK;
}

sdm_status check_opts(sdm_ctx *c, const sdm_opts *o) {
    if (!o) return fail(c, SDM_EINVAL, "opts is NULL");
    if (o->sstp_cond < 1 || o->sstp_coal < 1) return fail(c, SDM_EINVAL, "substep counts must be >= 1");
    if (o->coal_adapt < 0) return fail(c, SDM_EINVAL, "coal_adapt must be >= 0");
    if (!(o->RH_max > 0.0)) return fail(c, SDM_EINVAL, "RH_max must be positive");
    return SDM_OK;
}

}  // namespace

void sdm::sdm_set_global_error(const std::string &msg) { g_init_err = msg; }

// ---------------------------------------------------------------- ABI
extern "C" {

const char *sdm_last_error(const sdm_ctx *c) { return c ? c->err.c_str() : g_init_err.c_str(); }

sdm_status sdm_init(const sdm_opts_init *oi, sdm_arr th, sdm_arr rv, sdm_arr rhod, sdm_arr rhoCx,
                    sdm_arr rhoCy, sdm_arr rhoCz, void *stream, sdm_ctx **out) {
    if (!oi || !out) return fail(nullptr, SDM_EINVAL, "opts and out must not be NULL");
    *out = nullptr;
    {
        const char *fa = getenv("SDM_FAIL_ALLOC");
        g_fail_alloc = fa ? atoi(fa) : 0;
    }
    if (oi->backend != SDM_BACKEND_CUDA)
        return fail(nullptr, SDM_EINVAL, "only the CUDA back-end exists (no CPU fallback)");
    if (oi->nx < 0 || oi->ny < 0 || oi->nz < 0) return fail(nullptr, SDM_EINVAL, "negative cell count");
    if (oi->ny > 0 && (oi->nx == 0 || oi->nz == 0))
        return fail(nullptr, SDM_EINVAL, "a y dimension needs x and z dimensions");
    if (!(oi->dx > 0 && oi->dy > 0 && oi->dz > 0 && oi->dt > 0))
        return fail(nullptr, SDM_EINVAL, "dx, dy, dz and dt must be positive");
    if (oi->sd_conc < 1) return fail(nullptr, SDM_EINVAL, "sd_conc must be >= 1");
    if (oi->kernel != SDM_KERNEL_GEOMETRIC && oi->kernel != SDM_KERNEL_GOLOVIN && oi->kernel != SDM_KERNEL_LONG)
        return fail(nullptr, SDM_EINVAL, "unknown collision kernel");
    if (oi->precision != SDM_PRECISION_FP64 && oi->precision != SDM_PRECISION_MIXED)
        return fail(nullptr, SDM_EINVAL, "unknown precision mode");
    if (oi->cond_solver != SDM_SOLVER_BISECT && oi->cond_solver != SDM_SOLVER_FAST)
        return fail(nullptr, SDM_EINVAL, "unknown condensation solver");
    if (oi->cond_layout < SDM_COND_AUTO || oi->cond_layout > SDM_COND_STAGED)
        return fail(nullptr, SDM_EINVAL, "unknown condensation layout");
    if (oi->init_dist == SDM_INIT_LOGNORMAL) {
        if (oi->n_modes < 1 || oi->n_modes > kMaxModes || !oi->modes)
            return fail(nullptr, SDM_EINVAL, "lognormal initialisation needs 1..8 modes");
        for (int m = 0; m < oi->n_modes; ++m)
            if (!(oi->modes[m].rm > 0 && oi->modes[m].sigma > 1 && oi->modes[m].n_stp >= 0 &&
                  oi->modes[m].kappa > 0))
                return fail(nullptr, SDM_EINVAL, "invalid lognormal mode parameters");
    } else if (oi->init_dist == SDM_INIT_EXPONENTIAL) {
        if (!(oi->exp_mean_volume > 0 && oi->exp_n0 > 0))
            return fail(nullptr, SDM_EINVAL, "exponential initialisation needs positive volume and n0");
    } else {
        return fail(nullptr, SDM_EINVAL, "unknown initial distribution");
    }
    if (!th.data_zero || !rv.data_zero || !rhod.data_zero)
        return fail(nullptr, SDM_EINVAL, "th, rv and rhod are required");

    int ndev = 0;
    cudaError_t e = cudaGetDeviceCount(&ndev);
    if (e != cudaSuccess || ndev == 0)
        return fail(nullptr, SDM_ECUDA, std::string("no usable CUDA device: ") + cudaGetErrorString(e));

    sdm_ctx *c = new sdm_ctx();
    c->oi = *oi;
    if (oi->init_dist == SDM_INIT_LOGNORMAL) c->modes.assign(oi->modes, oi->modes + oi->n_modes);
    c->oi.modes = nullptr;
    cudaGetDevice(&c->device);
    Grid &g = c->grid;
    g.nx = oi->nx;
    g.ny = oi->ny;
    g.nz = oi->nz;
    g.NX = g.nx > 0 ? g.nx : 1;
    g.NY = g.ny > 0 ? g.ny : 1;
    g.NZ = g.nz > 0 ? g.nz : 1;
    g.dx = oi->dx;
    g.dy = oi->dy;
    g.dz = oi->dz;
    g.dt = oi->dt;
    g.dV = oi->dx * oi->dy * oi->dz;
    g.x_open = oi->x_open && oi->nx > 0 ? 1 : 0;
    const int64_t ncell = (int64_t)g.NX * g.NY * g.NZ;
    if (ncell > (1LL << 30)) {
        free_ctx(c);
        return fail(nullptr, SDM_EINVAL, "too many cells");
    }
    g.n_cells = (int)ncell;
    // distinct kappa groups, in order of first appearance
    if (oi->init_dist == SDM_INIT_LOGNORMAL) {
        for (const auto &m : c->modes) {
            bool seen = false;
            for (double k : c->gkappa) seen |= (k == m.kappa);
            if (!seen) c->gkappa.push_back(m.kappa);
        }
        for (double k : c->gkappa) {
            double lo, hi;
            if (!rd_range(c, k, &lo, &hi)) {
                free_ctx(c);
                return fail(nullptr, SDM_EINVAL, "no dry radius in [1 nm, 10 um] has multiplicity >= 1");
            }
            c->lnr_min.push_back(lo);
            c->lnr_max.push_back(hi);
        }
    } else {
        c->gkappa.push_back(0.0);
    }
    c->G = (int)c->gkappa.size();
    if (oi->sd_reserve < 0) {
        free_ctx(c);
        return fail(nullptr, SDM_EINVAL, "sd_reserve must be >= 0");
    }
    c->n_sd = ncell * c->G * oi->sd_conc + oi->sd_reserve;
    if (c->n_sd >= (1LL << 32) - 1) {
        free_ctx(c);
        return fail(nullptr, SDM_EINVAL, "more than 2^32 - 2 super-droplets");
    }
    if (stream) {
        c->stream = (cudaStream_t)stream;
    } else {
        e = cudaStreamCreateWithFlags(&c->stream, cudaStreamNonBlocking);
        if (e != cudaSuccess) {
            free_ctx(c);
            return fail(nullptr, SDM_ECUDA, "stream creation failed");
        }
        c->own_stream = true;
    }
    const size_t n = (size_t)c->n_sd, nc = (size_t)ncell;
    e = cudaSuccess;
    for (int b = 0; b < 2 && e == cudaSuccess; ++b) {
        SdArrays &s = c->buf[b];
        s = SdArrays{};
        if (e == cudaSuccess) e = dalloc(&s.N, n);
        if (e == cudaSuccess) e = dalloc(&s.rw2, n);
        if (e == cudaSuccess) e = dalloc(&s.rd3, n);
        if (e == cudaSuccess) e = dalloc(&s.kappa, n);
        if (e == cudaSuccess && g.nx > 0) e = dalloc(&s.x, n);
        if (e == cudaSuccess && g.ny > 0) e = dalloc(&s.y, n);
        if (e == cudaSuccess && g.nz > 0) e = dalloc(&s.z, n);
        if (e == cudaSuccess) e = dalloc(&s.uid, n);
    }
    size_t npow2 = 1;
    while (npow2 < n) npow2 <<= 1;
    if (e == cudaSuccess) e = dalloc(&c->newcell, n);
    if (e == cudaSuccess) e = dalloc(&c->slot, n);
    if (e == cudaSuccess) e = dalloc(&c->perm, n);
    if (e == cudaSuccess) e = dalloc(&c->count, nc + 1);
    if (e == cudaSuccess) e = dalloc(&c->offset, nc + 1);
    if (e == cudaSuccess) e = dalloc(&c->bigcells, nc);
    if (e == cudaSuccess && (int64_t)c->G * c->oi.sd_conc > kBigCellCap) e = dalloc(&c->huge, 6 * n);
    if (e == cudaSuccess) e = dalloc(&c->th, nc);
    if (e == cudaSuccess) e = dalloc(&c->rv, nc);
    if (e == cudaSuccess) e = dalloc(&c->rhod, nc);
    if (e == cudaSuccess) e = dalloc(&c->amb, 2 * nc);
    if (e == cudaSuccess) e = dalloc(&c->outbuf, nc);
    if (e == cudaSuccess) e = dalloc(&c->scan_tmp, nc / 1024 + 2);
    c->rc_tmp_bytes = 2 * npow2 * sizeof(SortRec);
    if (e == cudaSuccess) e = cudaMalloc(&c->rc_tmp, c->rc_tmp_bytes);
    if (e == cudaSuccess) e = cudaMalloc(&c->rc_sel, 4096);
    if (e == cudaSuccess) e = dalloc(&c->dstats, 1);
    if (e == cudaSuccess) e = cudaMallocHost((void **)&c->hstats, sizeof(DevStats));
    if (e == cudaSuccess) e = cudaEventCreateWithFlags(&c->done_event, cudaEventDisableTiming);
    if (e != cudaSuccess) {
        const bool oom = e == cudaErrorMemoryAllocation;
        std::string msg = std::string("allocation failed: ") + cudaGetErrorString(e);
        cudaGetLastError();
        free_ctx(c);
        return fail(nullptr, oom ? SDM_ENOMEM : SDM_ECUDA, msg);
    }
    memset(c->hstats, 0, sizeof(DevStats));
    cudaMemsetAsync(c->dstats, 0, sizeof(DevStats), c->stream);
    // Eulerian fields
    sdm_status st = field_in(c, c->th, th, -1, "th");
    if (st == SDM_OK) st = field_in(c, c->rv, rv, -1, "rv");
    if (st == SDM_OK) st = field_in(c, c->rhod, rhod, -1, "rhod");
    const sdm_arr *C[3] = {&rhoCx, &rhoCy, &rhoCz};
    const int dims[3] = {g.nx, g.ny, g.nz};
    for (int d = 0; d < 3 && st == SDM_OK; ++d) {
        if (!C[d]->data_zero || dims[d] == 0) continue;
        int shape[3];
        const int nd = field_shape(c, d, shape);
        int64_t tot = 1;
        for (int q = 0; q < nd; ++q) tot *= shape[q];
        if (cudaMalloc(&c->rhoC[d], tot * 8) != cudaSuccess) {
            st = SDM_ENOMEM;
            c->err = "Courant field allocation failed";
            break;
        }
        st = field_in(c, c->rhoC[d], *C[d], d, "rhoC");
    }
    if (st == SDM_OK) {
        e = launch_init(c);
        if (e == cudaSuccess) e = launch_ambient(c);
        // the reserved slots sit apart from the per-cell ranges: regroup first
        c->layout_dirty = c->oi.sd_reserve > 0;
        if (e == cudaSuccess) e = cudaStreamSynchronize(c->stream);
        if (e != cudaSuccess) {
            st = SDM_ECUDA;
            c->err = std::string("initialisation: ") + cudaGetErrorString(e);
        }
    }
    if (st != SDM_OK) {
        std::string msg = c->err;
        free_ctx(c);
        return fail(nullptr, st, msg);
    }
    g_fail_alloc = 0;
    *out = c;
    return SDM_OK;
}

sdm_status sdm_destroy(sdm_ctx *c) {
    if (!c) return SDM_OK;
    cudaStreamSynchronize(c->stream);
    free_ctx(c);
    return SDM_OK;
}

// the caller's rho_d C fields into the context's edge arrays (allocated on
// first use); absent arrays and absent dimensions are skipped
static sdm_status courant_in(sdm_ctx *c, const sdm_arr &rhoCx, const sdm_arr &rhoCy, const sdm_arr &rhoCz) {
    const sdm_arr *C[3] = {&rhoCx, &rhoCy, &rhoCz};
    const int dims[3] = {c->grid.nx, c->grid.ny, c->grid.nz};
    for (int d = 0; d < 3; ++d) {
        if (!C[d]->data_zero || dims[d] == 0) continue;
        if (!c->rhoC[d]) {
            int shape[3];
            const int nd = field_shape(c, d, shape);
            int64_t tot = 1;
            for (int q = 0; q < nd; ++q) tot *= shape[q];
            CK(cudaMalloc(&c->rhoC[d], tot * 8), "Courant allocation");
        }
        if (sdm_status s = field_in(c, c->rhoC[d], *C[d], d, "rhoC")) return s;
    }
    return SDM_OK;
}

sdm_status sdm_euler_step(sdm_ctx *c, const sdm_euler_opts *o, sdm_arr th, sdm_arr rv, sdm_arr rhoCx,
                          sdm_arr rhoCy, sdm_arr rhoCz) {
    if (!c || !o) return fail(c, SDM_EINVAL, "NULL argument");
    if (c->async_in_flight) return fail(c, SDM_ESTATE, "euler_step called before sdm_wait of step_async");
    if (!th.data_zero || !rv.data_zero) return fail(c, SDM_EINVAL, "th and rv are required");
    if (o->relax && (!o->th0 || !o->rv0 || !(o->tau_rlx > 0.0) || !(o->z_rlx > 0.0)))
        return fail(c, SDM_EINVAL, "relaxation needs th0, rv0 and positive tau_rlx, z_rlx");
    const int nz = c->grid.NZ;
    if (!c->euler_tmp) CK(cudaMalloc(&c->euler_tmp, 8 * (size_t)c->grid.n_cells), "Eulerian scratch");
    if (!c->euler_prof) CK(cudaMalloc(&c->euler_prof, 16 * (size_t)nz), "Eulerian scratch");
    Phase ph(c, PH_EULER);
    struct EulerCount {  // the field copies' launches count as the Eulerian step's too
        sdm_ctx *c;
        uint64_t l0;
        ~EulerCount() {
            c->tacc.euler_launches += c->tacc.launches - l0;
            c->tacc.launches = l0;
        }
    } count_guard{c, c->tacc.launches};
    if (sdm_status s = field_in(c, c->th, th, -1, "th")) return s;
    if (sdm_status s = field_in(c, c->rv, rv, -1, "rv")) return s;
    if (o->advect)
        if (sdm_status s = courant_in(c, rhoCx, rhoCy, rhoCz)) return s;
    if (o->relax) {
        CK(cudaMemcpyAsync(c->euler_prof, o->th0, 8 * (size_t)nz, cudaMemcpyHostToDevice, c->stream), "profiles");
        CK(cudaMemcpyAsync(c->euler_prof + nz, o->rv0, 8 * (size_t)nz, cudaMemcpyHostToDevice, c->stream),
           "profiles");
    }
    double *f[2] = {c->th, c->rv};
    for (int q = 0; q < 2; ++q) {
        if (o->advect) {
            CK(cudaMemcpyAsync(c->euler_tmp, f[q], 8 * (size_t)c->grid.n_cells, cudaMemcpyDeviceToDevice,
                               c->stream),
               "Eulerian copy");
            CK(launch_upwind(c->euler_tmp, f[q], c->rhod, rhoCx.data_zero ? c->rhoC[0] : nullptr,
                             rhoCy.data_zero ? c->rhoC[1] : nullptr, rhoCz.data_zero ? c->rhoC[2] : nullptr,
                             c->grid, c->stream),
               "upwind");
            c->tacc.launches += 1;
        }
        if (o->relax) {
            CK(launch_relax(f[q], c->euler_prof + q * nz, c->grid, o->tau_rlx, o->z_rlx, c->stream), "relax");
            c->tacc.launches += 1;
        }
    }
    if (sdm_status s = field_out(c, th, c->th, "th")) return s;
    if (sdm_status s = field_out(c, rv, c->rv, "rv")) return s;
    if (!th.on_device || !rv.on_device) CK(cudaStreamSynchronize(c->stream), "euler_step");
    return SDM_OK;
}

sdm_status sdm_step_sync(sdm_ctx *c, const sdm_opts *o, sdm_arr th, sdm_arr rv, sdm_arr rhoCx,
                         sdm_arr rhoCy, sdm_arr rhoCz, sdm_arr rhod) {
    if (!c) return fail(nullptr, SDM_EINVAL, "NULL context");
    if (sdm_status s = check_opts(c, o)) return s;
    if (c->async_in_flight) return fail(c, SDM_ESTATE, "step_sync called before sdm_wait of step_async");
    if (!th.data_zero || !rv.data_zero) return fail(c, SDM_EINVAL, "th and rv are required");
    {
        Phase ph(c, PH_COPY);
        if (sdm_status s = field_in(c, c->th, th, -1, "th")) return s;
        if (sdm_status s = field_in(c, c->rv, rv, -1, "rv")) return s;
        if (rhod.data_zero)
            if (sdm_status s = field_in(c, c->rhod, rhod, -1, "rhod")) return s;
        if (sdm_status s = courant_in(c, rhoCx, rhoCy, rhoCz)) return s;
    }
    if (c->layout_dirty)
        if (sdm_status s = regroup(c)) return s;
    if (o->cond) {
        Phase ph(c, PH_COND);
        int nl = 0;
        CK(launch_condense(c, *o, &nl), "condensation");
        c->tacc.launches += nl;
        c->tacc.cond_launches++;
    }
    {
        Phase ph(c, PH_COPY);
        if (sdm_status s = field_out(c, th, c->th, "th")) return s;
        if (sdm_status s = field_out(c, rv, c->rv, "rv")) return s;
    }
    if (!th.on_device || !rv.on_device) {
        CK(cudaStreamSynchronize(c->stream), "step_sync");
        unsigned flags = 0;
        CK(cudaMemcpy(&flags, &c->dstats->flags, sizeof(unsigned), cudaMemcpyDeviceToHost), "flags");
        return check_flags(c, flags);
    }
    return SDM_OK;
}

}  // extern "C"

namespace {

// The first half of a step_async: recycling, advection, sedimentation.
sdm_status enqueue_transport(sdm_ctx *c, const sdm_opts *o) {
    if (c->layout_dirty)
        if (sdm_status s = regroup(c)) return s;
    if (c->known_zeros > 0 && recycle_small(c)) {  // one block, no count through the host
        Phase ph(c, PH_RECYCLE);
        CK(launch_recycle_small(c), "recycle");
        c->tacc.launches += 1;
    } else if (c->known_zeros > 0) {
        Phase ph(c, PH_RECYCLE);
        CK(launch_recycle_compact(c), "recycle compact");
        c->tacc.launches += 1;
        unsigned cnt[2];
        CK(cudaMemcpyAsync(cnt, &c->dstats->n_rc_zero, sizeof(cnt), cudaMemcpyDeviceToHost, c->stream),
           "recycle counts");
        CK(cudaStreamSynchronize(c->stream), "recycle counts");
        if (cnt[0] > 0 && cnt[1] > 0) CK(launch_recycle_apply(c, cnt[0], cnt[1]), "recycle");
    }
    {
        Phase ph(c, PH_MOVE);
        CK(launch_ambient(c), "ambient");
        CK(launch_move(c, *o), "move");
        c->tacc.launches += 2 + (o->adve && (c->rhoC[0] || c->rhoC[1] || c->rhoC[2]) ? 1 : 0);  // + k_courant
    }
    return SDM_OK;
}

// The second half: regrouping and coalescence.  After an export or import
// the cells and counting-sort slots are taken afresh from the positions.
sdm_status enqueue_coalesce(sdm_ctx *c, const sdm_opts *o) {
    if (c->layout_dirty) {
        Phase ph(c, PH_MOVE);
        const sdm_opts still{0, 0, 0, 0, 44.0, 1, 1};
        CK(launch_move(c, still), "cells");
        c->tacc.launches += 1;
        c->layout_dirty = false;
    }
    {
        Phase ph(c, PH_SORT);
        CK(launch_regroup(c), "scan");
        c->tacc.launches += 4;
    }
    {
        Phase ph(c, PH_COAL);
        CK(launch_coalesce(c, *o, o->coal != 0), "coalescence");
        c->tacc.launches += 2;
        c->tacc.coal_launches++;
    }
    c->cur ^= 1;
    c->step++;
    CK(cudaEventRecord(c->done_event, c->stream), "event");
    c->async_in_flight = true;
    return SDM_OK;
}

// a block of n super-droplets in device memory: dst itself, or a staging
// copy of a host block (alloc, and fill from the host when upload)
struct DevBlock {
    sdm_sd_block b{};
    void *mem = nullptr;
    ~DevBlock() { cudaFree(mem); }
};

cudaError_t device_block(sdm_ctx *c, const sdm_sd_block &host, int64_t n, bool upload, DevBlock &out) {
    if (host.on_device) {
        out.b = host;
        return cudaSuccess;
    }
    const size_t m = (size_t)(n > 0 ? n : 1);
    cudaError_t e = cudaMalloc(&out.mem, m * (8 + 4 + 6 * 8));
    if (e != cudaSuccess) return e;
    char *p = (char *)out.mem;
    out.b.N = (uint64_t *)p;
    p += 8 * m;
    double *d = (double *)p;
    out.b.rw2 = d;
    out.b.rd3 = d + m;
    out.b.kappa = d + 2 * m;
    out.b.x = d + 3 * m;
    out.b.y = d + 4 * m;
    out.b.z = d + 5 * m;
    out.b.uid = (uint32_t *)(d + 6 * m);
    out.b.on_device = 1;
    if (upload && n > 0) {
        const cudaMemcpyKind h2d = cudaMemcpyHostToDevice;
        e = cudaMemcpyAsync(out.b.N, host.N, 8 * n, h2d, c->stream);
        if (e == cudaSuccess) e = cudaMemcpyAsync(out.b.uid, host.uid, 4 * n, h2d, c->stream);
        if (e == cudaSuccess) e = cudaMemcpyAsync(out.b.rw2, host.rw2, 8 * n, h2d, c->stream);
        if (e == cudaSuccess) e = cudaMemcpyAsync(out.b.rd3, host.rd3, 8 * n, h2d, c->stream);
        if (e == cudaSuccess) e = cudaMemcpyAsync(out.b.kappa, host.kappa, 8 * n, h2d, c->stream);
        if (e == cudaSuccess) e = cudaMemcpyAsync(out.b.x, host.x, 8 * n, h2d, c->stream);
        if (e == cudaSuccess && c->grid.ny > 0) e = cudaMemcpyAsync(out.b.y, host.y, 8 * n, h2d, c->stream);
        if (e == cudaSuccess && c->grid.nz > 0) e = cudaMemcpyAsync(out.b.z, host.z, 8 * n, h2d, c->stream);
    }
    return e;
}

bool block_complete(const sdm_ctx *c, const sdm_sd_block &b) {
    return b.N && b.uid && b.rw2 && b.rd3 && b.kappa && b.x && (c->grid.ny == 0 || b.y) && (c->grid.nz == 0 || b.z);
}

}  // namespace

extern "C" {

sdm_status sdm_step_async(sdm_ctx *c, const sdm_opts *o) {
    if (!c) return fail(nullptr, SDM_EINVAL, "NULL context");
    if (sdm_status s = check_opts(c, o)) return s;
    if (c->async_in_flight) return fail(c, SDM_ESTATE, "step_async called twice without sdm_wait");
    if (c->transported) return fail(c, SDM_ESTATE, "step_async with a transport pending (sdm_step_coalesce)");
    if (sdm_status s = enqueue_transport(c, o)) return s;
    return enqueue_coalesce(c, o);
}

sdm_status sdm_step_transport(sdm_ctx *c, const sdm_opts *o) {
    if (!c) return fail(nullptr, SDM_EINVAL, "NULL context");
    if (sdm_status s = check_opts(c, o)) return s;
    if (c->async_in_flight) return fail(c, SDM_ESTATE, "step_transport before sdm_wait of the previous step");
    if (c->transported) return fail(c, SDM_ESTATE, "step_transport twice without sdm_step_coalesce");
    if (sdm_status s = enqueue_transport(c, o)) return s;
    c->transported = true;
    return SDM_OK;
}

sdm_status sdm_step_coalesce(sdm_ctx *c, const sdm_opts *o) {
    if (!c) return fail(nullptr, SDM_EINVAL, "NULL context");
    if (sdm_status s = check_opts(c, o)) return s;
    if (!c->transported) return fail(c, SDM_ESTATE, "step_coalesce without sdm_step_transport");
    c->transported = false;
    return enqueue_coalesce(c, o);
}

sdm_status sdm_export_leavers(sdm_ctx *c, sdm_sd_block dst, int64_t cap, int64_t *n_out) {
    if (!c || !n_out) return fail(c, SDM_EINVAL, "NULL argument");
    *n_out = 0;
    if (!c->grid.x_open) return fail(c, SDM_EINVAL, "export_leavers needs an x_open context");
    if (c->async_in_flight) return fail(c, SDM_ESTATE, "export while a step is in flight");
    if (c->layout_dirty && !c->transported)
        if (sdm_status s = regroup(c)) return s;
    uint32_t cnt = 0;
    CK(launch_exchange_count(c, 1, &cnt), "leavers");
    *n_out = cnt;
    if ((int64_t)cnt > cap) return fail(c, SDM_ENOMEM, "the block holds fewer super-droplets than leave");
    if (cnt == 0) return SDM_OK;
    if (!block_complete(c, dst)) return fail(c, SDM_EINVAL, "a block array is NULL");
    DevBlock db;
    CK(device_block(c, dst, cnt, false, db), "export staging");
    CK(launch_export(c, db.b), "export");
    if (!dst.on_device) {
        const cudaMemcpyKind d2h = cudaMemcpyDeviceToHost;
        CK(cudaMemcpyAsync(dst.N, db.b.N, 8 * (size_t)cnt, d2h, c->stream), "export copy");
        CK(cudaMemcpyAsync(dst.uid, db.b.uid, 4 * (size_t)cnt, d2h, c->stream), "export copy");
        CK(cudaMemcpyAsync(dst.rw2, db.b.rw2, 8 * (size_t)cnt, d2h, c->stream), "export copy");
        CK(cudaMemcpyAsync(dst.rd3, db.b.rd3, 8 * (size_t)cnt, d2h, c->stream), "export copy");
        CK(cudaMemcpyAsync(dst.kappa, db.b.kappa, 8 * (size_t)cnt, d2h, c->stream), "export copy");
        CK(cudaMemcpyAsync(dst.x, db.b.x, 8 * (size_t)cnt, d2h, c->stream), "export copy");
        if (c->grid.ny > 0) CK(cudaMemcpyAsync(dst.y, db.b.y, 8 * (size_t)cnt, d2h, c->stream), "export copy");
        if (c->grid.nz > 0) CK(cudaMemcpyAsync(dst.z, db.b.z, 8 * (size_t)cnt, d2h, c->stream), "export copy");
    }
    CK(cudaStreamSynchronize(c->stream), "export");
    c->known_zeros += cnt;
    c->layout_dirty = true;
    return SDM_OK;
}

sdm_status sdm_import(sdm_ctx *c, sdm_sd_block src, int64_t n) {
    if (!c) return fail(nullptr, SDM_EINVAL, "NULL context");
    if (n < 0) return fail(c, SDM_EINVAL, "n must be >= 0");
    if (c->async_in_flight) return fail(c, SDM_ESTATE, "import while a step is in flight");
    if (n == 0) return SDM_OK;
    if (!block_complete(c, src)) return fail(c, SDM_EINVAL, "a block array is NULL");
    if (c->layout_dirty && !c->transported)
        if (sdm_status s = regroup(c)) return s;
    DevBlock db;
    CK(device_block(c, src, n, true, db), "import staging");
    unsigned bad = 0;
    CK(launch_block_check(c, db.b, n, &bad), "import check");
    if (bad)
        return fail(c, SDM_EINVAL, "an arriving super-droplet has N = 0, an id >= 2^31 or a position outside the domain");
    uint32_t free_slots = 0;
    CK(launch_exchange_count(c, 0, &free_slots), "free slots");
    if ((int64_t)free_slots < n) return fail(c, SDM_ENOMEM, "fewer free slots (N = 0) than arrivals");
    CK(launch_import(c, db.b, n), "import");
    CK(cudaStreamSynchronize(c->stream), "import");
    c->known_zeros = free_slots - (uint64_t)n;
    c->layout_dirty = true;
    return SDM_OK;
}

sdm_status sdm_wait(sdm_ctx *c, double timeout_s, double *rainfall_out) {
    if (!c) return fail(nullptr, SDM_EINVAL, "NULL context");
    if (c->async_in_flight) {
        const auto t0 = std::chrono::steady_clock::now();
        for (;;) {
            const cudaError_t q = cudaEventQuery(c->done_event);
            if (q == cudaSuccess) break;
            if (q != cudaErrorNotReady) return cuda_fail(c, q, "wait");
            const double el =
                std::chrono::duration<double>(std::chrono::steady_clock::now() - t0).count();
            if (timeout_s >= 0 && el > timeout_s)
                return fail(c, SDM_ETIMEOUT, "step_async still running at the deadline");
            std::this_thread::sleep_for(std::chrono::microseconds(20));
        }
        c->async_in_flight = false;
    }
    if (sdm_status s = pull_stats(c)) return s;
    c->known_zeros = c->mirror.n_zero;
    if (rainfall_out) *rainfall_out = c->mirror.rainfall;
    return check_flags(c, c->mirror.flags);
}

sdm_status sdm_diag_rng(sdm_ctx *c, int wet, double r_min, double r_max) {
    if (!c) return fail(nullptr, SDM_EINVAL, "NULL context");
    if (!(r_min <= r_max)) return fail(c, SDM_EINVAL, "r_min must not exceed r_max");
    c->diag_wet = wet ? 1 : 0;
    c->diag_rmin = r_min;
    c->diag_rmax = r_max;
    c->rng_set = true;
    return SDM_OK;
}

sdm_status sdm_diag_mom(sdm_ctx *c, int k) {
    if (!c) return fail(nullptr, SDM_EINVAL, "NULL context");
    if (!c->rng_set) return fail(c, SDM_ESTATE, "diag_mom before diag_rng");
    if (k < 0 || k > 8) return fail(c, SDM_EINVAL, "moment order must be 0..8");
    if (c->layout_dirty)
        if (sdm_status s = regroup(c)) return s;
    Phase ph(c, PH_DIAG);
    CK(launch_moments(c, k), "moments");
    c->tacc.launches += 1;
    return SDM_OK;
}

sdm_status sdm_diag_sd_conc(sdm_ctx *c) {
    if (!c) return fail(nullptr, SDM_EINVAL, "NULL context");
    if (c->layout_dirty)
        if (sdm_status s = regroup(c)) return s;
    Phase ph(c, PH_DIAG);
    CK(launch_sd_conc(c), "sd_conc");
    c->tacc.launches += 1;
    return SDM_OK;
}

sdm_status sdm_diag_ambient(sdm_ctx *c, int what) {
    if (!c) return fail(nullptr, SDM_EINVAL, "NULL context");
    if (what < 0 || what > 3) return fail(c, SDM_EINVAL, "what must be 0 (T), 1 (p), 2 (rho_vs) or 3 (RH)");
    Phase ph(c, PH_DIAG);
    CK(launch_cond_ambient(c, what), "ambient");
    c->tacc.launches += 1;
    return SDM_OK;
}

sdm_status sdm_diag_spectrum(sdm_ctx *c, int wet, const double *edges, int n_bins, int k, double *dst,
                             int dst_on_device) {
    if (!c) return fail(nullptr, SDM_EINVAL, "NULL context");
    if (!edges || !dst) return fail(c, SDM_EINVAL, "NULL argument");
    if (n_bins < 1 || n_bins > sdm::kMaxSpectrumBins) return fail(c, SDM_EINVAL, "n_bins must be 1..256");
    if (k < 0 || k > 8) return fail(c, SDM_EINVAL, "moment order must be 0..8");
    if (!(edges[0] >= 0.0)) return fail(c, SDM_EINVAL, "bin edges are radii: edges[0] must be >= 0");
    for (int b = 0; b < n_bins; ++b)
        if (!(edges[b] < edges[b + 1])) return fail(c, SDM_EINVAL, "bin edges must increase strictly");
    if (c->layout_dirty)
        if (sdm_status s = regroup(c)) return s;
    if (n_bins > c->spec_cap) {
        CK(cudaStreamSynchronize(c->stream), "spectrum buffer");
        cudaFree(c->spec_buf);
        c->spec_buf = nullptr;
        c->spec_cap = 0;
        CK(cudaMalloc(&c->spec_buf, sizeof(double) * (size_t)n_bins * (size_t)c->grid.n_cells), "spectrum buffer");
        if (!c->spec_edges)
            CK(cudaMalloc(&c->spec_edges, sizeof(double) * (sdm::kMaxSpectrumBins + 1)), "spectrum buffer");
        c->spec_cap = n_bins;
    }
    Phase ph(c, PH_DIAG);
    CK(cudaMemcpyAsync(c->spec_edges, edges, sizeof(double) * (size_t)(n_bins + 1), cudaMemcpyHostToDevice,
                       c->stream),
       "spectrum edges");
    CK(launch_spectrum(c, wet ? 1 : 0, n_bins, k), "spectrum");
    c->tacc.launches += 1;
    CK(cudaMemcpyAsync(dst, c->spec_buf, sizeof(double) * (size_t)n_bins * (size_t)c->grid.n_cells,
                       dst_on_device ? cudaMemcpyDeviceToDevice : cudaMemcpyDeviceToHost, c->stream),
       "spectrum copy");
    if (!dst_on_device) CK(cudaStreamSynchronize(c->stream), "spectrum copy");
    return SDM_OK;
}

sdm_status sdm_outbuf(sdm_ctx *c, double *dst, int dst_on_device) {
    if (!c || !dst) return fail(c, SDM_EINVAL, "NULL argument");
    CK(cudaMemcpyAsync(dst, c->outbuf, sizeof(double) * c->grid.n_cells,
                       dst_on_device ? cudaMemcpyDeviceToDevice : cudaMemcpyDeviceToHost, c->stream),
       "outbuf");
    if (!dst_on_device) CK(cudaStreamSynchronize(c->stream), "outbuf");
    return SDM_OK;
}

sdm_status sdm_sizes(const sdm_ctx *c, int64_t *n_sd, int64_t *n_cells) {
    if (!c) return fail(nullptr, SDM_EINVAL, "NULL context");
    if (n_sd) *n_sd = c->n_sd;
    if (n_cells) *n_cells = c->grid.n_cells;
    return SDM_OK;
}

static void *attr_ptr(sdm_ctx *c, int attr, size_t *esz) {
    SdArrays &s = c->buf[c->cur];
    *esz = 8;
    switch (attr) {
        case SDM_ATTR_N: return s.N;
        case SDM_ATTR_RW2: return s.rw2;
        case SDM_ATTR_RD3: return s.rd3;
        case SDM_ATTR_KAPPA: return s.kappa;
        case SDM_ATTR_X: return s.x;
        case SDM_ATTR_Y: return s.y;
        case SDM_ATTR_Z: return s.z;
        case SDM_ATTR_UID: *esz = 4; return s.uid;
        default: return nullptr;
    }
}

sdm_status sdm_get_attr(sdm_ctx *c, int attr, void *dst, int64_t n) {
    if (!c || !dst) return fail(c, SDM_EINVAL, "NULL argument");
    if (n != c->n_sd) return fail(c, SDM_EINVAL, "n must equal the number of super-droplets");
    if (c->layout_dirty)
        if (sdm_status s = regroup(c)) return s;
    size_t esz;
    void *p = attr_ptr(c, attr, &esz);
    if (!p) return fail(c, SDM_EINVAL, "unknown attribute or absent dimension");
    CK(cudaMemcpyAsync(dst, p, esz * n, cudaMemcpyDeviceToHost, c->stream), "get_attr");
    CK(cudaStreamSynchronize(c->stream), "get_attr");
    return SDM_OK;
}

sdm_status sdm_set_attr(sdm_ctx *c, int attr, const void *src, int64_t n) {
    if (!c || !src) return fail(c, SDM_EINVAL, "NULL argument");
    if (n != c->n_sd) return fail(c, SDM_EINVAL, "n must equal the number of super-droplets");
    if (c->async_in_flight) return fail(c, SDM_ESTATE, "set_attr while step_async is in flight");
    // no regroup here even when positions were set: a restore writes every
    // attribute in one storage order, and regrouping between two of its
    // calls would permute the slots under it; the next use regroups
    size_t esz;
    void *p = attr_ptr(c, attr, &esz);
    if (!p) return fail(c, SDM_EINVAL, "unknown attribute or absent dimension");
    CK(cudaMemcpyAsync(p, src, esz * n, cudaMemcpyHostToDevice, c->stream), "set_attr");
    CK(cudaStreamSynchronize(c->stream), "set_attr");
    if (attr == SDM_ATTR_X || attr == SDM_ATTR_Y || attr == SDM_ATTR_Z) c->layout_dirty = true;
    if (attr == SDM_ATTR_N) c->known_zeros = 1;  // recount at the next step
    return SDM_OK;
}

sdm_status sdm_get_fields(sdm_ctx *c, double *th, double *rv) {
    if (!c) return fail(nullptr, SDM_EINVAL, "NULL context");
    if (th) CK(cudaMemcpyAsync(th, c->th, 8 * c->grid.n_cells, cudaMemcpyDeviceToHost, c->stream), "fields");
    if (rv) CK(cudaMemcpyAsync(rv, c->rv, 8 * c->grid.n_cells, cudaMemcpyDeviceToHost, c->stream), "fields");
    CK(cudaStreamSynchronize(c->stream), "fields");
    return SDM_OK;
}

sdm_status sdm_get_step(const sdm_ctx *c, uint64_t *step) {
    if (!c || !step) return fail(nullptr, SDM_EINVAL, "NULL argument");
    *step = c->step;
    return SDM_OK;
}

sdm_status sdm_set_step(sdm_ctx *c, uint64_t step) {
    if (!c) return fail(nullptr, SDM_EINVAL, "NULL context");
    if (c->async_in_flight) return fail(c, SDM_ESTATE, "set_step while step_async is in flight");
    c->step = step;
    return SDM_OK;
}

sdm_status sdm_get_stats(sdm_ctx *c, sdm_stats *out) {
    if (!c || !out) return fail(c, SDM_EINVAL, "NULL argument");
    if (sdm_status s = pull_stats(c)) return s;
    const DevStats &m = c->mirror;
    out->n_pairs = m.n_pairs;
    out->n_coll = m.n_coll;
    out->n_pgt1 = m.n_pgt1;
    out->n_recycled = c->host_recycled + m.n_recycled;  // the large path counts on the host, the small on the device
    out->n_euler = m.n_euler;
    out->n_fallback = m.n_fallback;
    out->n_steps = c->step;
    out->n_zero = m.n_zero;
    double mp;
    memcpy(&mp, &m.max_p_bits, sizeof(mp));
    out->max_p = mp;
    out->rainfall = m.rainfall;
    out->n_coal_substeps = m.n_coal_substeps;
    return SDM_OK;
}

sdm_status sdm_timing_enable(sdm_ctx *c, int on) {
    if (!c) return fail(nullptr, SDM_EINVAL, "NULL context");
    c->timing = on != 0;
    return SDM_OK;
}

sdm_status sdm_get_timing(sdm_ctx *c, sdm_timing *out, int reset) {
    if (!c || !out) return fail(c, SDM_EINVAL, "NULL argument");
    CK(cudaStreamSynchronize(c->stream), "timing");
    for (auto &t : c->timers) {
        float ms = 0.f;
        cudaEventElapsedTime(&ms, t.a, t.b);
        double *dst = nullptr;
        switch (t.phase) {
            case PH_COND: dst = &c->tacc.cond_ms; break;
            case PH_RECYCLE: dst = &c->tacc.recycle_ms; break;
            case PH_MOVE: dst = &c->tacc.move_ms; break;
            case PH_SORT: dst = &c->tacc.sort_ms; break;
            case PH_COAL: dst = &c->tacc.coal_ms; break;
            case PH_DIAG: dst = &c->tacc.diag_ms; break;
            case PH_EULER: dst = &c->tacc.euler_ms; break;
            default: dst = &c->tacc.copy_ms; break;
        }
        *dst += ms;
        c->event_pool.push_back(t.a);
        c->event_pool.push_back(t.b);
    }
    c->timers.clear();
    *out = c->tacc;
    if (reset) memset(&c->tacc, 0, sizeof(c->tacc));
    return SDM_OK;
}

}  // extern "C"
