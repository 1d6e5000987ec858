// Batched ensembles of 0D members (boxes and adiabatic parcels, the parcel
// framework of the paper's particles_t with no spatial dimension) advanced
// together: one set of launches per step for all members, whatever their
// sizes, captured into one CUDA graph.
//
// Every member is an independent simulation: its random numbers come from
// Philox under its own key (seed, 0) with counters (id, substep, own step,
// stream), its ids run 0..n-1, and nothing it computes depends on the other
// members - so a member gives the same result alone and in any mix.
//
// Layout: the members' super-droplets are packed back to back (member-major,
// ids ascending), with a member index per super-droplet.  Condensation works
// on tiles that never straddle two members: per substep one launch solves
// every super-droplet and reduces each tile, a second sums each member's
// tiles in a fixed order and updates its r_v and theta (eq. rhov_update).
// Coalescence per substep: keys, a stable radix sort by (member, key), then
// one thread per pair.  Parcels conserve their dry-air mass: when rho_d is
// given for a step, the volume becomes m_d / rho_d.
#include <math.h>
#include <string.h>

#include <algorithm>
#include <chrono>
#include <thread>

#include "sdm_internal.cuh"

namespace sdm {

template <class K>
cudaError_t radix_sort_pairs(K *key_a, uint32_t *val_a, uint32_t *aux_a, K *key_b, uint32_t *val_b,
                             uint32_t *aux_b, int64_t n, int key_bytes, int aux_bytes, uint32_t *hist,
                             uint32_t *scan_tmp, cudaStream_t st);

constexpr int kEnsMaxModes = 4;

struct MemberInitDev {
    int init_dist, n_modes;
    double lrm[kEnsMaxModes], lsig[kEnsMaxModes], n_stp[kEnsMaxModes];
    double kappa, lmin, lmax, exp_mean_volume, exp_n0;
};

}  // namespace sdm

struct sdm_ens {
    sdm_ens_opts eo;
    int device = 0;
    cudaStream_t stream = nullptr;
    bool own_stream = false;
    int64_t cap_sd = 0;
    int cap_members = 0;
    // host mirror of the member table (members in packing order)
    std::vector<sdm_member> params;
    std::vector<int32_t> ids;          // public id of each packed member
    std::vector<char> alive;
    std::vector<sdm::MemberDev> mhost;
    int32_t next_id = 0;
    int64_t n_sd = 0;
    bool dirty_pack = false;
    // device state
    sdm::SdArrays s[2]{};
    int cur = 0;
    uint32_t *mem[2] = {nullptr, nullptr};   // member index per super-droplet
    sdm::MemberDev *mdev = nullptr;
    sdm::MemberInitDev *minit = nullptr;
    uint32_t *tile_member = nullptr, *tile_beg = nullptr, *tile_end = nullptr;
    double *tile_sum = nullptr;
    int n_tiles = 0;
    // coalescence sort buffers
    unsigned long long *key[2] = {nullptr, nullptr};
    uint32_t *val[2] = {nullptr, nullptr}, *aux[2] = {nullptr, nullptr};
    uint32_t *hist = nullptr, *scan_tmp = nullptr;
    unsigned long long *acc = nullptr;
    uint32_t *live = nullptr;  // live super-droplets per member (coalescence substep)
    double *rhod_dev = nullptr, *rhod_pin = nullptr;
    double *outbuf = nullptr;
    sdm::DevStats *dstats = nullptr, *hstats = nullptr;
    cudaEvent_t done = nullptr;
    bool in_flight = false;
    // graph of one step
    cudaGraphExec_t graph = nullptr;
    sdm_opts graph_opts{};
    bool graph_rhod = false;
    bool use_graph = false;
    // tuning: tile size and threads per block of the condensation launch
    int tile = 256, cond_threads = 128, pair_threads = 256;
    size_t reserved = 0;  // device bytes the arena holds from creation to destruction
    std::string err;
};

namespace sdm {

// ---------------------------------------------------------------- kernels
__global__ void k_ens_init(SdArrays s, uint32_t *mem, const MemberDev *M, const MemberInitDev *MI,
                           uint32_t m_first, uint32_t m_last, uint32_t q0, uint32_t q1) {
    const uint32_t q = q0 + blockIdx.x * blockDim.x + threadIdx.x;
    if (q >= q1) return;
    // the member holding q (m_last - m_first is small; linear search)
    uint32_t m = m_first;
    while (m + 1 < m_last && M[m + 1].off <= q) ++m;
    const MemberDev &md = M[m];
    const MemberInitDev &p = MI[m];
    const uint32_t uid = q - md.off;
    mem[q] = m;
    s.uid[q] = uid;
    const u64x4 w = philox4x64(uid, 0, 0, kStreamInit, md.seed, 0);
    if (p.init_dist == SDM_INIT_EXPONENTIAL) {
        const double V = -p.exp_mean_volume * log(u01(w.v[3]));
        const double r = cbrt(3.0 * V / (4.0 * phys::pi));
        s.rw2[q] = r * r;
        s.rd3[q] = 0.0;
        s.kappa[q] = 0.0;
        const double nn = floor(p.exp_n0 * md.dV / md.n + 0.5);
        s.N[q] = nn < 1.0 ? 1ull : (unsigned long long)nn;
        return;
    }
    const double lnr = __dadd_rn(p.lmin, __dmul_rn(u01(w.v[3]), p.lmax - p.lmin));
    const double rd = exp(lnr);
    const double rd3 = rd * rd * rd;
    const double dlnr = (p.lmax - p.lmin) / md.n;
    double nl = 0.0;
    for (int k = 0; k < p.n_modes; ++k) {
        const double q2 = (lnr - p.lrm[k]) / p.lsig[k];
        nl = __dadd_rn(nl, __dmul_rn(p.n_stp[k] / (sqrt(2.0 * phys::pi) * p.lsig[k]), exp(-0.5 * q2 * q2)));
    }
    const double nn = floor(nl * dlnr * md.dV * md.rhod / phys::rho_stp + 0.5);
    s.N[q] = nn < 1.0 ? 1ull : (unsigned long long)nn;
    s.rd3[q] = rd3;
    s.kappa[q] = p.kappa;
    const Thermo t = thermo_eval(md.th, md.rv, md.rhod, 44.0);
    double RH = t.rho_v / t.rho_vs;
    if (RH >= 1.0) RH = 0.95;
    // equilibrium wet radius (zero growth rate), bisection as in k_init.cu
    const double rd2 = rd2_of(rd3);
    double out = rd2;
    if (p.kappa > 0.0 && RH > 0.0 && RH < 1.0 && rd3 > 0.0) {
        const double A = 2.0 * phys::sigma_w / (phys::R_v * t.T * phys::rho_w);
        const double rhi = cbrt(rd3 * (1.0 - RH * (1.0 - p.kappa)) / (1.0 - RH));
        double lo = rd2, hi = rhi * rhi;
        for (int it = 0; it < 200; ++it) {
            if (hi - lo <= 0x1p-52 * hi) break;
            const double mid = 0.5 * (lo + hi);
            if (!(mid > lo && mid < hi)) break;
            const double r = sqrt(mid), r3 = mid * r;
            const double S = (r3 - rd3) / (r3 - rd3 * (1.0 - p.kappa)) * exp(A / r);
            if (S > RH) hi = mid;
            else lo = mid;
        }
        out = 0.5 * (lo + hi);
    }
    s.rw2[q] = out;
}

__global__ void k_ens_rhod(MemberDev *M, const double *rhod, int nm) {
    const int m = blockIdx.x * blockDim.x + threadIdx.x;
    if (m >= nm || rhod[m] == M[m].rhod) return;
    M[m].rhod = rhod[m];
    M[m].dV = M[m].md / rhod[m];
}

// recycling inside each member: the k-th zero (id order = storage order)
// takes the k-th donor in (N descending, id ascending) order among N >= 2;
// at most kEnsRecyclePerStep per member and step (the rest wait a step)
constexpr int kEnsRecyclePerStep = 64;

__global__ void k_ens_recycle(SdArrays s, MemberDev *M, DevStats *st) {
    const MemberDev &md = M[blockIdx.x];
    // the coalescence kernel counts every multiplicity that reaches zero
    if (md.zeros == 0) return;
    __shared__ unsigned s_z;
    __shared__ unsigned long long s_best;
    __shared__ uint32_t s_bestq;
    __shared__ uint32_t s_zq[kEnsRecyclePerStep], s_dq[kEnsRecyclePerStep];
    __shared__ unsigned long long s_prevN;
    __shared__ uint32_t s_prevq;
    // fast path: count the zeros
    if (threadIdx.x == 0) s_z = 0;
    __syncthreads();
    unsigned zc = 0;
    for (uint32_t q = threadIdx.x; q < md.n; q += blockDim.x) zc += s.N[md.off + q] == 0;
    zc = __reduce_add_sync(0xffffffffu, zc);
    if ((threadIdx.x & 31) == 0 && zc) atomicAdd(&s_z, zc);
    __syncthreads();
    const unsigned total = s_z;
    if (total == 0) {
        if (threadIdx.x == 0) M[blockIdx.x].zeros = 0;
        return;
    }
    // the first zeros in storage (= id) order, found by one warp in sequence
    if (threadIdx.x < 32) {
        const int lane = threadIdx.x;
        unsigned found = 0;
        for (uint32_t base = 0; base < md.n && found < kEnsRecyclePerStep; base += 32) {
            const uint32_t q = base + lane;
            const bool z = q < md.n && s.N[md.off + q] == 0;
            const unsigned bal = __ballot_sync(0xffffffffu, z);
            if (z) {
                const unsigned r = found + __popc(bal & ((1u << lane) - 1u));
                if (r < kEnsRecyclePerStep) s_zq[r] = q;
            }
            found += __popc(bal);
        }
        if (lane == 0) s_z = min(found, (unsigned)kEnsRecyclePerStep);
    }
    __syncthreads();
    const unsigned nz = s_z;
    if (threadIdx.x == 0) {
        s_prevN = ~0ull;
        s_prevq = 0;
    }
    __syncthreads();
    unsigned nd = 0;
    for (unsigned k = 0; k < nz; ++k) {
        // next donor: the largest (N, -id) below the previous one, N >= 2
        if (threadIdx.x == 0) {
            s_best = 0;
            s_bestq = 0xffffffffu;
        }
        __syncthreads();
        const unsigned long long pN = s_prevN;
        const uint32_t pq = s_prevq;
        unsigned long long bestN = 0;
        uint32_t bestq = 0xffffffffu;
        for (uint32_t q = threadIdx.x; q < md.n; q += blockDim.x) {
            const unsigned long long N = s.N[md.off + q];
            if (N < 2) continue;
            const bool below = N < pN || (N == pN && q > pq);
            if (!below) continue;
            if (N > bestN || (N == bestN && q < bestq)) {
                bestN = N;
                bestq = q;
            }
        }
        // block arg-max: pack (N, ~q) into one word for each candidate
        for (int o = 16; o > 0; o >>= 1) {
            const unsigned long long oN = __shfl_xor_sync(0xffffffffu, bestN, o);
            const uint32_t oq = __shfl_xor_sync(0xffffffffu, bestq, o);
            if (oN > bestN || (oN == bestN && oq < bestq)) {
                bestN = oN;
                bestq = oq;
            }
        }
        if ((threadIdx.x & 31) == 0 && bestN > 0) {
            // serialise the warp leaders through one lock-free compare loop
            atomicMax(&s_best, bestN);
        }
        __syncthreads();
        if ((threadIdx.x & 31) == 0 && bestN > 0 && bestN == s_best) atomicMin(&s_bestq, bestq);
        __syncthreads();
        if (s_best < 2) break;
        if (threadIdx.x == 0) {
            s_dq[k] = s_bestq;
            s_prevN = s_best;
            s_prevq = s_bestq;
        }
        __syncthreads();
        nd = k + 1;
    }
    const unsigned np = min(nz, nd);
    for (unsigned k = threadIdx.x; k < np; k += blockDim.x) {
        const uint32_t z = md.off + s_zq[k], d = md.off + s_dq[k];
        s.rw2[z] = s.rw2[d];
        s.rd3[z] = s.rd3[d];
        s.kappa[z] = s.kappa[d];
        const unsigned long long Nd = s.N[d];
        s.N[z] = Nd / 2;
        s.N[d] = Nd - Nd / 2;
    }
    if (threadIdx.x == 0) {
        M[blockIdx.x].zeros = total - np;
        if (np) atomicAdd(&st->n_recycled, (unsigned long long)np);
    }
}

// one warp per member: lane l adds tiles l, l + 32, ... and the warp
// combines the lanes in a fixed tree (the same order in any ensemble)
__global__ void k_ens_cond_update(MemberDev *M, const double *tile_sum, int nm, EnsCondParams p,
                                  DevStats *st) {
    const int64_t m64 = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const int lane = threadIdx.x & 31;
    if (m64 >= nm) return;  // whole warps leave together
    MemberDev &md = M[m64];
    double sum = 0.0;
    for (uint32_t t = lane; t < md.ntiles; t += 32) sum += tile_sum[md.tile0 + t];
    for (int o = 16; o > 0; o >>= 1) sum += __shfl_xor_sync(0xffffffffu, sum, o);
    if (lane) return;
    const Thermo t = thermo_eval(md.th, md.rv, md.rhod, p.RH_max);
    const double drv = -4.0 * phys::pi * phys::rho_w / (3.0 * md.dV * md.rhod) * sum;
    md.rv = t.rv + drv;
    md.th = t.th + drv * t.dth_drv;
    if (!isfinite(md.rv) || !isfinite(md.th)) atomicOr(&st->flags, kFlagNumeric);
}

struct EnsCoalParams {
    double dt;
    int sstp, kernel, mixed;
    double golovin_b;
    int multi;
};

// sort keys of one coalescence substep: word 0 of the pairing draw (its
// 31 leading bits in mixed precision, so that the inactive key 0xFFFFFFFF
// sorts strictly after every live one); the live super-droplets of each
// member are counted on the way (block-aggregated atomics: members are
// stored contiguously, so a block rarely spans more than one)
template <class K>
__global__ void k_ens_keys(const SdArrays s, const uint32_t *mem, const MemberDev *M, int64_t n, int sub,
                           K *key, uint32_t *val, uint32_t *aux, unsigned long long *acc, uint32_t *act) {
    __shared__ uint32_t s_cnt;
    const int64_t q0 = (int64_t)blockIdx.x * blockDim.x;
    const int64_t q = q0 + threadIdx.x;
    const bool ok = q < n;
    const uint32_t m0 = mem[q0];
    if (threadIdx.x == 0) s_cnt = 0;
    __syncthreads();
    uint32_t m = 0xffffffffu;
    bool live = false;
    if (ok) {
        m = mem[q];
        const MemberDev &md = M[m];
        K k = (K)~0ull;
        if (s.N[q] > 0) {
            const u64x4 w = philox4x64(s.uid[q], (uint64_t)sub, md.step, kStreamCoal, md.seed, 0);
            k = sizeof(K) == 4 ? (K)(w.v[0] >> 33) : (K)w.v[0];
            acc[q] = w.v[1];
            live = true;
        }
        key[q] = k;
        val[q] = (uint32_t)q;
        aux[q] = m;
    }
    const unsigned peers = __match_any_sync(0xffffffffu, m);
    const unsigned cnt = __popc(__ballot_sync(0xffffffffu, live) & peers);
    if (ok && cnt && (threadIdx.x & 31) == (unsigned)(__ffs(peers) - 1)) {
        if (m == m0) atomicAdd(&s_cnt, cnt);
        else atomicAdd(&act[m], cnt);
    }
    __syncthreads();
    if (threadIdx.x == 0 && s_cnt) atomicAdd(&act[m0], s_cnt);
}

__global__ void k_ens_pairs(SdArrays s, MemberDev *M, const uint32_t *aux, const uint32_t *val,
                            const unsigned long long *acc, const uint32_t *live, int64_t n, EnsCoalParams p,
                            DevStats *st) {
    const int64_t q = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    unsigned long long npair = 0, ncoll = 0, ngt1 = 0;
    double mp = 0.0;
    if (q < n) {
        const uint32_t m = aux[q];
        const MemberDev &md = M[m];
        const uint32_t j = (uint32_t)(q - md.off);
        const uint32_t act = live[m];
        if ((j & 1u) == 0 && j + 1 < act) {
            const uint32_t a = val[q], b = val[q + 1];
            const double scale = pair_scale(act);
            const double dtpp = p.dt / p.sstp;
            const double Ra = s.rw2[a], Rb = s.rw2[b];
            const unsigned long long Na = s.N[a], Nb = s.N[b];
            const unsigned long long Nmax = Na > Nb ? Na : Nb;
            double P;
            struct {
                double nu, cX;
            } t{md.nu, md.cX};
            if (p.mixed) {
                float K;
                if (p.kernel == SDM_KERNEL_GOLOVIN) {
                    const float fa = (float)Ra, fb = (float)Rb;
                    K = (float)p.golovin_b * (4.0f / 3.0f * (float)phys::pi) * (fa * sqrtf(fa) + fb * sqrtf(fb));
                } else {
                    const float ra = sqrtf((float)Ra), rb = sqrtf((float)Rb);
                    const float va = vterm_f((float)Ra, (float)t.nu, (float)t.cX);
                    const float vb = vterm_f((float)Rb, (float)t.nu, (float)t.cX);
                    K = (float)phys::pi * (ra + rb) * (ra + rb) * fabsf(va - vb);
                    if (p.kernel == SDM_KERNEL_LONG) K = long_Ef(ra, rb) * K;
                }
                const float Pf = (float)Nmax * K * (float)dtpp / (float)md.dV * (float)scale;
                P = Pf;
            } else {
                double K;
                if (p.kernel == SDM_KERNEL_GOLOVIN) {
                    const double Va = 4.0 / 3.0 * phys::pi * Ra * sqrt(Ra);
                    const double Vb = 4.0 / 3.0 * phys::pi * Rb * sqrt(Rb);
                    K = p.golovin_b * (Va + Vb);
                } else {
                    const double ra = sqrt(Ra), rb = sqrt(Rb);
                    const double dv = fabs(vterm(Ra, t.nu, t.cX) - vterm(Rb, t.nu, t.cX));
                    K = phys::pi * (ra + rb) * (ra + rb) * dv;
                    if (p.kernel == SDM_KERNEL_LONG) K = long_E(ra, rb) * K;
                }
                P = (double)Nmax * K * dtpp / md.dV * scale;
            }
            const unsigned long long gam = n_events(P, acc[a], Nmax, Na > Nb ? Nb : Na, p.multi, p.mixed);
            npair = 1;
            ngt1 = P > 1.0;
            mp = P;
            if (gam) {  // gamma events, as collide() in the single-context kernels
                const uint32_t L = Na >= Nb ? a : b, S = L == a ? b : a;
                const unsigned long long NS = s.N[S];
                s.N[L] -= gam * NS;
                if (s.N[L] == 0) atomicAdd(&M[m].zeros, 1u);  // recycled at the next step
                const double g = (double)gam;
                const double rwS = s.rw2[S], rwL = s.rw2[L];
                const double r = cbrt(rwS * sqrt(rwS) + g * (rwL * sqrt(rwL)));
                s.rw2[S] = r * r;
                const double dS = s.rd3[S], dL = g * s.rd3[L], m3 = dS + dL;
                if (m3 > 0.0) s.kappa[S] = (s.kappa[S] * dS + s.kappa[L] * dL) / m3;
                s.rd3[S] = m3;
                ncoll = 1;
            }
        }
    }
    const unsigned a1 = __reduce_add_sync(0xffffffffu, (unsigned)npair);
    const unsigned a2 = __reduce_add_sync(0xffffffffu, (unsigned)ncoll);
    const unsigned a3 = __reduce_add_sync(0xffffffffu, (unsigned)ngt1);
    for (int o = 16; o > 0; o >>= 1) mp = fmax(mp, __shfl_xor_sync(0xffffffffu, mp, o));
    if ((threadIdx.x & 31) == 0) {
        if (a1) atomicAdd(&st->n_pairs, (unsigned long long)a1);
        if (a2) atomicAdd(&st->n_coll, (unsigned long long)a2);
        if (a3) atomicAdd(&st->n_pgt1, (unsigned long long)a3);
        if (mp > 0.0) atomicMax(&st->max_p_bits, (unsigned long long)__double_as_longlong(mp));
    }
}

// air viscosity and Best-number factor of each member for this step's
// terminal velocities (from theta, r_v, rho_d after condensation)
__global__ void k_ens_ambient(MemberDev *M, int nm) {
    const int m = blockIdx.x * blockDim.x + threadIdx.x;
    if (m >= nm) return;
    const Thermo t = thermo_eval(M[m].th, M[m].rv, M[m].rhod, 44.0);
    M[m].nu = t.nu;
    M[m].cX = t.cX;
}

__global__ void k_ens_step_done(MemberDev *M, int nm) {
    const int m = blockIdx.x * blockDim.x + threadIdx.x;
    if (m < nm) M[m].step++;
}

__global__ void k_ens_moments(const SdArrays s, const MemberDev *M, int wet, double rmin, double rmax,
                              int k, double *out) {
    const MemberDev &md = M[blockIdx.x];
    double sum = 0.0;
    for (uint32_t q = threadIdx.x; q < md.n; q += blockDim.x) {
        const uint32_t i = md.off + q;
        const double r = wet ? sqrt(s.rw2[i]) : cbrt(s.rd3[i]);
        if (!(r >= rmin && r <= rmax)) continue;
        double pw = 1.0;
        for (int e = 0; e < k; ++e) pw *= r;
        sum += (double)s.N[i] * pw;
    }
    __shared__ double part[32];
    for (int o = 16; o > 0; o >>= 1) sum += __shfl_xor_sync(0xffffffffu, sum, o);
    if ((threadIdx.x & 31) == 0) part[threadIdx.x >> 5] = sum;
    __syncthreads();
    if (threadIdx.x == 0) {
        double t = 0.0;
        for (int w = 0; w < (int)(blockDim.x >> 5); ++w) t += part[w];
        out[blockIdx.x] = t / (md.rhod * md.dV);
    }
}

// move each live member's super-droplets to its new packed range
__global__ void k_ens_repack(SdArrays src, SdArrays dst, const uint32_t *mem_src, uint32_t *mem_dst,
                             const uint32_t *old_off, const uint32_t *new_off, const int *new_index,
                             int64_t n_old) {
    const int64_t q = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (q >= n_old) return;
    const uint32_t m = mem_src[q];
    const int nm = new_index[m];
    if (nm < 0) return;
    const uint32_t d = new_off[nm] + (uint32_t)(q - old_off[m]);
    dst.N[d] = src.N[q];
    dst.rw2[d] = src.rw2[q];
    dst.rd3[d] = src.rd3[q];
    dst.kappa[d] = src.kappa[q];
    dst.uid[d] = src.uid[q];
    mem_dst[d] = (uint32_t)nm;
}

}  // namespace sdm

// ---------------------------------------------------------------- host side
namespace {
using namespace sdm;

sdm_status efail(sdm_ens *e, sdm_status s, const std::string &m) {
    if (e) e->err = m;
    else sdm_set_global_error(m);
    return s;
}

#define ECK(call, where)                                                                     \
    do {                                                                                     \
        cudaError_t e_ = (call);                                                             \
        if (e_ != cudaSuccess) return efail(e, SDM_ECUDA, std::string(where) + ": " + cudaGetErrorString(e_)); \
    } while (0)

int aux_bytes_for(int nm) { return nm <= 256 ? 1 : (nm <= 65536 ? 2 : 3); }

int n_members(const sdm_ens *e) { return (int)e->mhost.size(); }

int64_t max_tiles(const sdm_ens *e) { return e->cap_sd / 128 + e->cap_members + 1; }

// refresh the host mirror of the fields the device evolves
sdm_status pull_members(sdm_ens *e) {
    const int nm = n_members(e);
    ECK(cudaStreamSynchronize(e->stream), "sync");
    if (nm) ECK(cudaMemcpy(e->mhost.data(), e->mdev, sizeof(MemberDev) * nm, cudaMemcpyDeviceToHost), "members");
    return SDM_OK;
}

sdm_status push_tables(sdm_ens *e) {
    const int nm = n_members(e);
    std::vector<uint32_t> tm, tb, te;
    for (int m = 0; m < nm; ++m) {
        MemberDev &md = e->mhost[m];
        md.tile0 = (uint32_t)tm.size();
        for (uint32_t b = 0; b < md.n; b += (uint32_t)e->tile) {
            tm.push_back((uint32_t)m);
            tb.push_back(md.off + b);
            te.push_back(md.off + std::min<uint32_t>(b + (uint32_t)e->tile, md.n));
        }
        md.ntiles = (uint32_t)tm.size() - md.tile0;
    }
    if ((int64_t)tm.size() > max_tiles(e)) return efail(e, SDM_EINVAL, "too many tiles for the arena");
    e->n_tiles = (int)tm.size();
    if (e->n_tiles) {
        ECK(cudaMemcpy(e->tile_member, tm.data(), 4 * tm.size(), cudaMemcpyHostToDevice), "tiles");
        ECK(cudaMemcpy(e->tile_beg, tb.data(), 4 * tb.size(), cudaMemcpyHostToDevice), "tiles");
        ECK(cudaMemcpy(e->tile_end, te.data(), 4 * te.size(), cudaMemcpyHostToDevice), "tiles");
    }
    if (nm) ECK(cudaMemcpy(e->mdev, e->mhost.data(), sizeof(MemberDev) * nm, cudaMemcpyHostToDevice), "members");
    if (e->graph) {
        cudaGraphExecDestroy(e->graph);
        e->graph = nullptr;
    }
    return SDM_OK;
}

// drop retired members and pack the survivors from offset 0
sdm_status repack(sdm_ens *e, std::vector<MemberInitDev> &minit) {
    const int nm = n_members(e);
    std::vector<uint32_t> old_off(nm), new_off;
    std::vector<int> new_index(nm, -1);
    std::vector<MemberDev> nh;
    std::vector<sdm_member> np;
    std::vector<int32_t> nid;
    std::vector<char> nal;
    std::vector<MemberInitDev> ni;
    uint32_t end = 0;
    for (int m = 0; m < nm; ++m) {
        old_off[m] = e->mhost[m].off;
        if (!e->alive[m]) continue;
        new_index[m] = (int)nh.size();
        MemberDev md = e->mhost[m];
        md.off = end;
        new_off.push_back(end);
        end += md.n;
        nh.push_back(md);
        np.push_back(e->params[m]);
        nid.push_back(e->ids[m]);
        nal.push_back(1);
        ni.push_back(minit[m]);
    }
    if (e->n_sd > 0 && !nh.empty()) {
        uint32_t *d_old = nullptr, *d_new = nullptr;
        int *d_idx = nullptr;
        ECK(cudaMallocAsync(&d_old, 4 * nm, e->stream), "repack");
        ECK(cudaMallocAsync(&d_new, 4 * nh.size(), e->stream), "repack");
        ECK(cudaMallocAsync(&d_idx, 4 * nm, e->stream), "repack");
        ECK(cudaMemcpyAsync(d_old, old_off.data(), 4 * nm, cudaMemcpyHostToDevice, e->stream), "repack");
        ECK(cudaMemcpyAsync(d_new, new_off.data(), 4 * nh.size(), cudaMemcpyHostToDevice, e->stream), "repack");
        ECK(cudaMemcpyAsync(d_idx, new_index.data(), 4 * nm, cudaMemcpyHostToDevice, e->stream), "repack");
        k_ens_repack<<<grid_for(e->n_sd, 256), 256, 0, e->stream>>>(e->s[e->cur], e->s[e->cur ^ 1],
                                                                    e->mem[e->cur], e->mem[e->cur ^ 1],
                                                                    d_old, d_new, d_idx, e->n_sd);
        ECK(cudaGetLastError(), "repack");
        cudaFreeAsync(d_old, e->stream);
        cudaFreeAsync(d_new, e->stream);
        cudaFreeAsync(d_idx, e->stream);
        ECK(cudaStreamSynchronize(e->stream), "repack");
        e->cur ^= 1;
    }
    e->mhost = nh;
    e->params = np;
    e->ids = nid;
    e->alive = nal;
    minit = ni;
    e->n_sd = end;
    e->dirty_pack = false;
    if (!minit.empty())
        ECK(cudaMemcpy(e->minit, minit.data(), sizeof(MemberInitDev) * minit.size(), cudaMemcpyHostToDevice),
            "init table");
    for (size_t m = 0; m < nh.size(); ++m) e->rhod_pin[m] = nh[m].rhod;
    return push_tables(e);
}

// One coalescence substep of every member: Philox keys, a stable radix sort
// by (member, key), one thread per pair.
sdm_status enqueue_coal_substep(sdm_ens *e, const EnsCoalParams &p, int ab, int sub, cudaStream_t st) {
    const int nm = n_members(e);
    const int64_t n = e->n_sd;
    ECK(cudaMemsetAsync(e->live, 0, 4 * (size_t)nm, st), "live counts");
    if (p.mixed) {
        uint32_t *k0 = reinterpret_cast<uint32_t *>(e->key[0]), *k1 = reinterpret_cast<uint32_t *>(e->key[1]);
        k_ens_keys<uint32_t><<<grid_for(n, 256), 256, 0, st>>>(e->s[e->cur], e->mem[e->cur], e->mdev, n, sub, k0,
                                                              e->val[0], e->aux[0], e->acc, e->live);
        ECK(radix_sort_pairs<uint32_t>(k0, e->val[0], e->aux[0], k1, e->val[1], e->aux[1], n, 4, ab, e->hist,
                                       e->scan_tmp, st),
            "sort");
    } else {
        k_ens_keys<unsigned long long><<<grid_for(n, 256), 256, 0, st>>>(e->s[e->cur], e->mem[e->cur], e->mdev, n, sub,
                                                                        e->key[0], e->val[0], e->aux[0], e->acc,
                                                                        e->live);
        ECK(radix_sort_pairs<unsigned long long>(e->key[0], e->val[0], e->aux[0], e->key[1], e->val[1], e->aux[1], n,
                                                 8, ab, e->hist, e->scan_tmp, st),
            "sort");
    }
    k_ens_pairs<<<grid_for(n, e->pair_threads), e->pair_threads, 0, st>>>(e->s[e->cur], e->mdev, e->aux[0],
                                                                           e->val[0], e->acc, e->live, n, p,
                                                                           e->dstats);
    return SDM_OK;
}

sdm_status enqueue_step(sdm_ens *e, const sdm_opts &o) {
    const int nm = n_members(e);
    if (nm == 0) return SDM_OK;
    cudaStream_t st = e->stream;
    ECK(cudaMemcpyAsync(e->rhod_dev, e->rhod_pin, 8 * nm, cudaMemcpyHostToDevice, st), "rhod");
    k_ens_rhod<<<grid_for(nm, 128), 128, 0, st>>>(e->mdev, e->rhod_dev, nm);
    k_ens_recycle<<<nm, 256, 0, st>>>(e->s[e->cur], e->mdev, e->dstats);
    const bool mixed = e->eo.precision == SDM_PRECISION_MIXED;
    if (o.cond) {
        EnsCondParams p{e->eo.dt, o.sstp_cond, e->eo.physics, e->eo.cond_solver, mixed ? 1 : 0, o.RH_max};
        for (int sub = 0; sub < o.sstp_cond; ++sub) {
            ECK(launch_ens_cond_tiles(e->s[e->cur], e->mdev, e->tile_member, e->tile_beg, e->tile_end,
                                      e->tile_sum, e->n_tiles, e->cond_threads, p, e->dstats, st),
                "condensation");
            k_ens_cond_update<<<grid_for((int64_t)nm * 32, 128), 128, 0, st>>>(e->mdev, e->tile_sum, nm, p,
                                                                                e->dstats);
        }
    }
    if (o.coal) {
        EnsCoalParams p{e->eo.dt, o.sstp_coal, e->eo.kernel, mixed ? 1 : 0, e->eo.golovin_b, o.coal_multi ? 1 : 0};
        const int ab = aux_bytes_for(nm);
        k_ens_ambient<<<grid_for(nm, 128), 128, 0, st>>>(e->mdev, nm);
        for (int sub = 0; sub < o.sstp_coal; ++sub)
            if (sdm_status s = enqueue_coal_substep(e, p, ab, sub, st)) return s;
    }
    k_ens_step_done<<<grid_for(nm, 128), 128, 0, st>>>(e->mdev, nm);
    ECK(cudaGetLastError(), "step");
    return SDM_OK;
}

int find_member(const sdm_ens *e, int32_t id) {
    for (size_t m = 0; m < e->ids.size(); ++m)
        if (e->ids[m] == id && e->alive[m]) return (int)m;
    return -1;
}

void free_ens(sdm_ens *e) {
    if (!e) return;
    for (int b = 0; b < 2; ++b) {
        cudaFree(e->s[b].N);
        cudaFree(e->s[b].rw2);
        cudaFree(e->s[b].rd3);
        cudaFree(e->s[b].kappa);
        cudaFree(e->s[b].uid);
        cudaFree(e->mem[b]);
        cudaFree(e->key[b]);
        cudaFree(e->val[b]);
        cudaFree(e->aux[b]);
    }
    cudaFree(e->mdev);
    cudaFree(e->minit);
    cudaFree(e->tile_member);
    cudaFree(e->tile_beg);
    cudaFree(e->tile_end);
    cudaFree(e->tile_sum);
    cudaFree(e->hist);
    cudaFree(e->scan_tmp);
    cudaFree(e->acc);
    cudaFree(e->live);
    cudaFree(e->rhod_dev);
    cudaFree(e->outbuf);
    cudaFree(e->dstats);
    if (e->hstats) cudaFreeHost(e->hstats);
    if (e->rhod_pin) cudaFreeHost(e->rhod_pin);
    if (e->graph) cudaGraphExecDestroy(e->graph);
    if (e->done) cudaEventDestroy(e->done);
    if (e->own_stream && e->stream) cudaStreamDestroy(e->stream);
    delete e;
}

}  // namespace

// host copies of the init tables, keyed by ensemble
#include <map>
static std::map<const sdm_ens *, std::vector<MemberInitDev>> g_minit;

extern "C" {

const char *sdm_ens_last_error(const sdm_ens *e) { return e ? e->err.c_str() : sdm_last_error(nullptr); }

sdm_status sdm_ens_create(const sdm_ens_opts *o, void *stream, sdm_ens **out) {
    if (!o || !out) return efail(nullptr, SDM_EINVAL, "opts and out must not be NULL");
    *out = nullptr;
    if (!(o->dt > 0) || o->max_sd < 1 || o->max_members < 1 || o->max_sd >= (1LL << 31))
        return efail(nullptr, SDM_EINVAL, "need dt > 0, 1 <= max_sd < 2^31, max_members >= 1");
    if (o->kernel != SDM_KERNEL_GEOMETRIC && o->kernel != SDM_KERNEL_GOLOVIN && o->kernel != SDM_KERNEL_LONG)
        return efail(nullptr, SDM_EINVAL, "unknown collision kernel");
    if (o->precision != SDM_PRECISION_FP64 && o->precision != SDM_PRECISION_MIXED)
        return efail(nullptr, SDM_EINVAL, "unknown precision mode");
    int ndev = 0;
    if (cudaGetDeviceCount(&ndev) != cudaSuccess || ndev == 0) {
        cudaGetLastError();
        return efail(nullptr, SDM_ECUDA, "no usable CUDA device");
    }
    sdm_ens *e = new sdm_ens();
    e->eo = *o;
    e->cap_sd = o->max_sd;
    e->cap_members = o->max_members;
    cudaGetDevice(&e->device);
    cudaError_t r = cudaSuccess;
    if (stream) e->stream = (cudaStream_t)stream;
    else {
        r = cudaStreamCreateWithFlags(&e->stream, cudaStreamNonBlocking);
        e->own_stream = true;
    }
    const size_t n = (size_t)e->cap_sd, nm = (size_t)e->cap_members;
    const int64_t tiles_rs = (e->cap_sd + kRsTileRecords - 1) / kRsTileRecords;
    auto A = [&](void **p, size_t bytes) {
        if (r == cudaSuccess) r = cudaMalloc(p, bytes);
        if (r == cudaSuccess) e->reserved += bytes;
    };
    for (int b = 0; b < 2; ++b) {
        A((void **)&e->s[b].N, 8 * n);
        A((void **)&e->s[b].rw2, 8 * n);
        A((void **)&e->s[b].rd3, 8 * n);
        A((void **)&e->s[b].kappa, 8 * n);
        A((void **)&e->s[b].uid, 4 * n);
        A((void **)&e->mem[b], 4 * n);
        A((void **)&e->key[b], 8 * n);
        A((void **)&e->val[b], 4 * n);
        A((void **)&e->aux[b], 4 * n);
    }
    A((void **)&e->mdev, sizeof(MemberDev) * nm);
    A((void **)&e->minit, sizeof(MemberInitDev) * nm);
    const size_t mt = (size_t)max_tiles(e);
    A((void **)&e->tile_member, 4 * mt);
    A((void **)&e->tile_beg, 4 * mt);
    A((void **)&e->tile_end, 4 * mt);
    A((void **)&e->tile_sum, 8 * mt);
    A((void **)&e->hist, 4 * (256 * (size_t)tiles_rs + 1));
    A((void **)&e->scan_tmp, 4 * (256 * (size_t)tiles_rs / 1024 + 4));
    A((void **)&e->acc, 8 * n);
    A((void **)&e->live, 4 * nm);
    A((void **)&e->rhod_dev, 8 * nm);
    A((void **)&e->outbuf, 8 * nm);
    A((void **)&e->dstats, sizeof(DevStats));
    if (r == cudaSuccess) r = cudaMallocHost((void **)&e->hstats, sizeof(DevStats));
    if (r == cudaSuccess) r = cudaMallocHost((void **)&e->rhod_pin, 8 * nm);
    if (r == cudaSuccess) r = cudaEventCreateWithFlags(&e->done, cudaEventDisableTiming);
    if (r == cudaSuccess) r = cudaMemset(e->dstats, 0, sizeof(DevStats));
    if (r != cudaSuccess) {
        const bool oom = r == cudaErrorMemoryAllocation;
        std::string msg = std::string("ensemble allocation: ") + cudaGetErrorString(r);
        cudaGetLastError();
        free_ens(e);
        return efail(nullptr, oom ? SDM_ENOMEM : SDM_ECUDA, msg);
    }
    g_minit[e].clear();
    *out = e;
    return SDM_OK;
}

sdm_status sdm_ens_memory(const sdm_ens *e, size_t *device_bytes, int64_t *cap_sd, int32_t *cap_members) {
    if (!e) return efail(nullptr, SDM_EINVAL, "NULL ensemble");
    if (device_bytes) *device_bytes = e->reserved;
    if (cap_sd) *cap_sd = e->cap_sd;
    if (cap_members) *cap_members = e->cap_members;
    return SDM_OK;
}

sdm_status sdm_ens_destroy(sdm_ens *e) {
    if (!e) return SDM_OK;
    cudaStreamSynchronize(e->stream);
    g_minit.erase(e);
    free_ens(e);
    return SDM_OK;
}

sdm_status sdm_ens_add(sdm_ens *e, const sdm_member *m, int32_t *id) {
    if (!e || !m || !id) return efail(e, SDM_EINVAL, "NULL argument");
    if (e->in_flight) return efail(e, SDM_ESTATE, "add while a step is in flight");
    if (m->n_sd < 1 || !(m->dV > 0) || !(m->rhod > 0))
        return efail(e, SDM_EINVAL, "member needs n_sd >= 1, dV > 0, rhod > 0");
    MemberInitDev mi{};
    mi.init_dist = m->init_dist;
    if (m->init_dist == SDM_INIT_LOGNORMAL) {
        if (m->n_modes < 1 || m->n_modes > kEnsMaxModes) return efail(e, SDM_EINVAL, "1..4 modes");
        for (int k = 0; k < m->n_modes; ++k) {
            if (m->modes[k].kappa != m->modes[0].kappa)
                return efail(e, SDM_EINVAL, "ensemble members take one kappa");
            if (!(m->modes[k].rm > 0 && m->modes[k].sigma > 1 && m->modes[k].n_stp >= 0))
                return efail(e, SDM_EINVAL, "invalid lognormal mode");
            mi.lrm[k] = log(m->modes[k].rm);
            mi.lsig[k] = log(m->modes[k].sigma);
            mi.n_stp[k] = m->modes[k].n_stp;
        }
        mi.n_modes = m->n_modes;
        mi.kappa = m->modes[0].kappa;
        std::vector<sdm_lognormal> modes(m->modes, m->modes + m->n_modes);
        if (!rd_range_modes(modes, mi.kappa, m->n_sd, m->dV, &mi.lmin, &mi.lmax))
            return efail(e, SDM_EINVAL, "no dry radius in [1 nm, 10 um] has multiplicity >= 1");
    } else if (m->init_dist == SDM_INIT_EXPONENTIAL) {
        if (!(m->exp_mean_volume > 0 && m->exp_n0 > 0)) return efail(e, SDM_EINVAL, "bad exponential spectrum");
        mi.exp_mean_volume = m->exp_mean_volume;
        mi.exp_n0 = m->exp_n0;
    } else {
        return efail(e, SDM_EINVAL, "unknown initial distribution");
    }
    int live = 0;
    int64_t live_sd = 0;
    for (size_t k = 0; k < e->mhost.size(); ++k)
        if (e->alive[k]) {
            live++;
            live_sd += e->mhost[k].n;
        }
    if (live_sd + m->n_sd > e->cap_sd || live + 1 > e->cap_members)
        return efail(e, SDM_ENOMEM, "the ensemble arena is full");
    auto &minit = g_minit[e];
    if (sdm_status s = pull_members(e)) return s;
    if (e->dirty_pack || e->n_sd + m->n_sd > e->cap_sd || (int)e->mhost.size() + 1 > e->cap_members)
        if (sdm_status s = repack(e, minit)) return s;
    MemberDev md{};
    md.off = (uint32_t)e->n_sd;
    md.n = (uint32_t)m->n_sd;
    md.dV = m->dV;
    md.md = m->rhod * m->dV;
    md.th = m->th;
    md.rv = m->rv;
    md.rhod = m->rhod;
    md.seed = m->seed;
    md.step = 0;
    const int idx = (int)e->mhost.size();
    e->mhost.push_back(md);
    e->params.push_back(*m);
    e->ids.push_back(e->next_id);
    e->alive.push_back(1);
    minit.push_back(mi);
    e->rhod_pin[idx] = m->rhod;
    e->n_sd += m->n_sd;
    ECK(cudaMemcpy(e->minit + idx, &mi, sizeof(mi), cudaMemcpyHostToDevice), "init table");
    if (sdm_status s = push_tables(e)) return s;
    const uint32_t q0 = md.off, q1 = md.off + md.n;
    k_ens_init<<<grid_for(q1 - q0, 256), 256, 0, e->stream>>>(e->s[e->cur], e->mem[e->cur], e->mdev, e->minit,
                                                              (uint32_t)idx, (uint32_t)idx + 1, q0, q1);
    ECK(cudaGetLastError(), "member init");
    ECK(cudaStreamSynchronize(e->stream), "member init");
    *id = e->next_id++;
    return SDM_OK;
}

sdm_status sdm_ens_remove(sdm_ens *e, int32_t id) {
    if (!e) return efail(nullptr, SDM_EINVAL, "NULL ensemble");
    if (e->in_flight) return efail(e, SDM_ESTATE, "remove while a step is in flight");
    const int m = find_member(e, id);
    if (m < 0) return efail(e, SDM_EINVAL, "no such member");
    e->alive[m] = 0;
    e->dirty_pack = true;
    return SDM_OK;
}

sdm_status sdm_ens_members(const sdm_ens *e, int32_t *ids, int32_t cap, int32_t *n, int64_t *n_sd) {
    if (!e) return efail(nullptr, SDM_EINVAL, "NULL ensemble");
    int32_t k = 0;
    int64_t tot = 0;
    for (size_t m = 0; m < e->ids.size(); ++m) {
        if (!e->alive[m]) continue;
        if (ids && k < cap) ids[k] = e->ids[m];
        k++;
        tot += e->mhost[m].n;
    }
    if (n) *n = k;
    if (n_sd) *n_sd = tot;
    return SDM_OK;
}

// field by field: a caller's struct may carry any bytes in its padding
static bool same_opts(const sdm_opts &a, const sdm_opts &b) {
    return a.adve == b.adve && a.sedi == b.sedi && a.cond == b.cond && a.coal == b.coal && a.RH_max == b.RH_max &&
           a.sstp_cond == b.sstp_cond && a.sstp_coal == b.sstp_coal && a.coal_multi == b.coal_multi &&
           a.coal_adapt == b.coal_adapt;
}

sdm_status sdm_ens_step(sdm_ens *e, const sdm_opts *o, const int32_t *ids, const double *rhod, int32_t n) {
    if (!e || !o) return efail(e, SDM_EINVAL, "NULL argument");
    if (e->in_flight) return efail(e, SDM_ESTATE, "step before sdm_ens_wait of the previous one");
    if (o->sstp_cond < 1 || o->sstp_coal < 1) return efail(e, SDM_EINVAL, "substep counts must be >= 1");
    if (o->coal_adapt != 0) return efail(e, SDM_EINVAL, "adaptive coalescence substeps: single contexts only");
    if (e->dirty_pack) {
        if (sdm_status s = pull_members(e)) return s;
        if (sdm_status s = repack(e, g_minit[e])) return s;
    }
    for (int32_t k = 0; k < n && ids && rhod; ++k) {
        const int m = find_member(e, ids[k]);
        if (m < 0 || !(rhod[k] > 0)) return efail(e, SDM_EINVAL, "bad member id or rho_d");
        e->rhod_pin[m] = rhod[k];
    }
    if (e->use_graph) {
        const bool same = e->graph && same_opts(e->graph_opts, *o);
        if (!same) {
            if (e->graph) cudaGraphExecDestroy(e->graph);
            e->graph = nullptr;
            cudaGraph_t g;
            ECK(cudaStreamBeginCapture(e->stream, cudaStreamCaptureModeThreadLocal), "capture");
            const sdm_status s = enqueue_step(e, *o);
            const cudaError_t ce = cudaStreamEndCapture(e->stream, &g);
            if (s != SDM_OK) return s;
            ECK(ce, "capture");
            ECK(cudaGraphInstantiate(&e->graph, g, 0), "instantiate");
            cudaGraphDestroy(g);
            e->graph_opts = *o;
        }
        ECK(cudaGraphLaunch(e->graph, e->stream), "graph launch");
    } else {
        if (sdm_status s = enqueue_step(e, *o)) return s;
    }
    ECK(cudaEventRecord(e->done, e->stream), "event");
    e->in_flight = true;
    return SDM_OK;
}

sdm_status sdm_ens_wait(sdm_ens *e, double timeout_s) {
    if (!e) return efail(nullptr, SDM_EINVAL, "NULL ensemble");
    if (!e->in_flight) return SDM_OK;
    const auto t0 = std::chrono::steady_clock::now();
    for (;;) {
        const cudaError_t q = cudaEventQuery(e->done);
        if (q == cudaSuccess) break;
        if (q != cudaErrorNotReady) return efail(e, SDM_ECUDA, cudaGetErrorString(q));
        const double el = std::chrono::duration<double>(std::chrono::steady_clock::now() - t0).count();
        if (timeout_s >= 0 && el > timeout_s) return efail(e, SDM_ETIMEOUT, "step still running at the deadline");
        std::this_thread::sleep_for(std::chrono::microseconds(20));
    }
    e->in_flight = false;
    unsigned flags = 0;
    ECK(cudaMemcpy(&flags, &e->dstats->flags, sizeof(unsigned), cudaMemcpyDeviceToHost), "flags");
    if (flags & kFlagNumeric) return efail(e, SDM_ENUMERIC, "a kernel produced a non-finite value");
    return SDM_OK;
}

sdm_status sdm_ens_moments(sdm_ens *e, int wet, double rmin, double rmax, int k, const int32_t *ids, double *out,
                           int32_t n) {
    if (!e || (n > 0 && (!ids || !out))) return efail(e, SDM_EINVAL, "NULL argument");
    if (k < 0 || k > 8) return efail(e, SDM_EINVAL, "moment order must be 0..8");
    const int nm = n_members(e);
    if (nm == 0) return SDM_OK;
    k_ens_moments<<<nm, 256, 0, e->stream>>>(e->s[e->cur], e->mdev, wet ? 1 : 0, rmin, rmax, k, e->outbuf);
    ECK(cudaGetLastError(), "moments");
    std::vector<double> all(nm);
    ECK(cudaMemcpyAsync(all.data(), e->outbuf, 8 * nm, cudaMemcpyDeviceToHost, e->stream), "moments");
    ECK(cudaStreamSynchronize(e->stream), "moments");
    for (int32_t q = 0; q < n; ++q) {
        const int m = find_member(e, ids[q]);
        if (m < 0) return efail(e, SDM_EINVAL, "no such member");
        out[q] = all[m];
    }
    return SDM_OK;
}

sdm_status sdm_ens_fields(sdm_ens *e, const int32_t *ids, double *th, double *rv, int32_t n) {
    if (!e) return efail(nullptr, SDM_EINVAL, "NULL ensemble");
    if (sdm_status s = pull_members(e)) return s;
    for (int32_t q = 0; q < n; ++q) {
        const int m = find_member(e, ids[q]);
        if (m < 0) return efail(e, SDM_EINVAL, "no such member");
        if (th) th[q] = e->mhost[m].th;
        if (rv) rv[q] = e->mhost[m].rv;
    }
    return SDM_OK;
}

sdm_status sdm_ens_get_attr(sdm_ens *e, int32_t id, int attr, void *dst, int64_t n) {
    if (!e || !dst) return efail(e, SDM_EINVAL, "NULL argument");
    const int m = find_member(e, id);
    if (m < 0) return efail(e, SDM_EINVAL, "no such member");
    if (e->dirty_pack) {
        if (sdm_status s = pull_members(e)) return s;
        if (sdm_status s = repack(e, g_minit[e])) return s;
    }
    const int mm = find_member(e, id);
    const MemberDev &md = e->mhost[mm];
    if (n != (int64_t)md.n) return efail(e, SDM_EINVAL, "n must equal the member's super-droplet count");
    const SdArrays &s = e->s[e->cur];
    const void *src = nullptr;
    size_t esz = 8;
    switch (attr) {
        case SDM_ATTR_N: src = s.N + md.off; break;
        case SDM_ATTR_RW2: src = s.rw2 + md.off; break;
        case SDM_ATTR_RD3: src = s.rd3 + md.off; break;
        case SDM_ATTR_KAPPA: src = s.kappa + md.off; break;
        case SDM_ATTR_UID: src = s.uid + md.off; esz = 4; break;
        default: return efail(e, SDM_EINVAL, "attribute not held by 0D members");
    }
    ECK(cudaMemcpyAsync(dst, src, esz * n, cudaMemcpyDeviceToHost, e->stream), "get_attr");
    ECK(cudaStreamSynchronize(e->stream), "get_attr");
    return SDM_OK;
}

sdm_status sdm_ens_use_graph(sdm_ens *e, int on) {
    if (!e) return efail(nullptr, SDM_EINVAL, "NULL ensemble");
    e->use_graph = on != 0;
    return SDM_OK;
}

sdm_status sdm_ens_autotune(sdm_ens *e, const sdm_opts *o, int *tile_out, int *threads_out,
                            int *pair_threads_out) {
    if (!e || !o) return efail(e, SDM_EINVAL, "NULL argument");
    if (e->in_flight) return efail(e, SDM_ESTATE, "autotune while a step is in flight");
    if (e->dirty_pack) {
        if (sdm_status s = pull_members(e)) return s;
        if (sdm_status s = repack(e, g_minit[e])) return s;
    }
    const int nm = n_members(e);
    if (nm == 0 || e->n_sd == 0) return efail(e, SDM_ESTATE, "no members to tune on");
    if (sdm_status s = pull_members(e)) return s;
    // keep the state: r_w^2 in a scratch buffer, the counters on the host
    ECK(cudaMemcpyAsync(e->key[1], e->s[e->cur].rw2, 8 * e->n_sd, cudaMemcpyDeviceToDevice, e->stream), "tune");
    DevStats saved;
    ECK(cudaMemcpyAsync(&saved, e->dstats, sizeof(DevStats), cudaMemcpyDeviceToHost, e->stream), "tune");
    ECK(cudaStreamSynchronize(e->stream), "tune");
    const int cand[][2] = {{128, 128}, {256, 128}, {256, 256}, {512, 128}, {512, 256}, {1024, 256}, {2048, 512}};
    const bool mixed = e->eo.precision == SDM_PRECISION_MIXED;
    EnsCondParams p{e->eo.dt, o->sstp_cond, e->eo.physics, e->eo.cond_solver, mixed ? 1 : 0, o->RH_max};
    cudaEvent_t a, b;
    cudaEventCreate(&a);
    cudaEventCreate(&b);
    float best = 1e30f;
    int bt = e->tile, bth = e->cond_threads;
    const int max_threads = ens_cond_max_threads(p);
    for (auto &c : cand) {
        if (c[1] > max_threads) continue;
        e->tile = c[0];
        e->cond_threads = c[1];
        if (sdm_status s = push_tables(e)) return s;
        float tot = 0.f;
        for (int rep = 0; rep < 4; ++rep) {
            ECK(cudaMemcpyAsync(e->s[e->cur].rw2, e->key[1], 8 * e->n_sd, cudaMemcpyDeviceToDevice, e->stream),
                "tune");
            cudaEventRecord(a, e->stream);
            ECK(launch_ens_cond_tiles(e->s[e->cur], e->mdev, e->tile_member, e->tile_beg, e->tile_end,
                                      e->tile_sum, e->n_tiles, e->cond_threads, p, e->dstats, e->stream),
                "tune");
            cudaEventRecord(b, e->stream);
            cudaEventSynchronize(b);
            float ms = 0.f;
            cudaEventElapsedTime(&ms, a, b);
            if (rep > 0) tot += ms;
        }
        if (tot < best) {
            best = tot;
            bt = c[0];
            bth = c[1];
        }
    }
    e->tile = bt;
    e->cond_threads = bth;
    ECK(cudaMemcpyAsync(e->s[e->cur].rw2, e->key[1], 8 * e->n_sd, cudaMemcpyDeviceToDevice, e->stream), "tune");
    if (sdm_status s = push_tables(e)) return s;
    // coalescence: the pair kernel's block size over one substep (keys, sort,
    // pairs), the state kept in the arena's second buffer and put back
    int bp = e->pair_threads;
    if (o->coal) {
        const SdArrays cur = e->s[e->cur], spare = e->s[e->cur ^ 1];
        const size_t n = (size_t)e->n_sd;
        auto save = [&](const SdArrays &from, const SdArrays &to) {
            cudaMemcpyAsync(to.N, from.N, 8 * n, cudaMemcpyDeviceToDevice, e->stream);
            cudaMemcpyAsync(to.rw2, from.rw2, 8 * n, cudaMemcpyDeviceToDevice, e->stream);
            cudaMemcpyAsync(to.rd3, from.rd3, 8 * n, cudaMemcpyDeviceToDevice, e->stream);
            return cudaMemcpyAsync(to.kappa, from.kappa, 8 * n, cudaMemcpyDeviceToDevice, e->stream);
        };
        ECK(save(cur, spare), "tune");
        EnsCoalParams cp{e->eo.dt, o->sstp_coal, e->eo.kernel, mixed ? 1 : 0, e->eo.golovin_b, o->coal_multi ? 1 : 0};
        const int ab = aux_bytes_for(nm);
        k_ens_ambient<<<grid_for(nm, 128), 128, 0, e->stream>>>(e->mdev, nm);
        float bestc = 1e30f;
        for (int pt : {64, 128, 256, 512}) {
            e->pair_threads = pt;
            float tot = 0.f;
            for (int rep = 0; rep < 4; ++rep) {
                ECK(save(spare, cur), "tune");
                cudaEventRecord(a, e->stream);
                if (sdm_status s = enqueue_coal_substep(e, cp, ab, 0, e->stream)) return s;
                cudaEventRecord(b, e->stream);
                cudaEventSynchronize(b);
                float ms = 0.f;
                cudaEventElapsedTime(&ms, a, b);
                if (rep > 0) tot += ms;
            }
            if (tot < bestc) {
                bestc = tot;
                bp = pt;
            }
        }
        e->pair_threads = bp;
        ECK(save(spare, cur), "tune");
    }
    cudaEventDestroy(a);
    cudaEventDestroy(b);
    ECK(cudaMemcpyAsync(e->dstats, &saved, sizeof(DevStats), cudaMemcpyHostToDevice, e->stream), "tune");
    ECK(cudaStreamSynchronize(e->stream), "tune");
    if (e->graph) {  // a captured step holds the old launch shapes
        cudaGraphExecDestroy(e->graph);
        e->graph = nullptr;
    }
    if (tile_out) *tile_out = bt;
    if (threads_out) *threads_out = bth;
    if (pair_threads_out) *pair_threads_out = bp;
    return SDM_OK;
}

sdm_status sdm_ens_stats(sdm_ens *e, sdm_stats *out) {
    if (!e || !out) return efail(e, SDM_EINVAL, "NULL argument");
    ECK(cudaMemcpyAsync(e->hstats, e->dstats, sizeof(DevStats), cudaMemcpyDeviceToHost, e->stream), "stats");
    ECK(cudaStreamSynchronize(e->stream), "stats");
    const DevStats &m = *e->hstats;
    memset(out, 0, sizeof(*out));
    out->n_pairs = m.n_pairs;
    out->n_coll = m.n_coll;
    out->n_pgt1 = m.n_pgt1;
    out->n_recycled = m.n_recycled;
    out->n_euler = m.n_euler;
    out->n_fallback = m.n_fallback;
    double mp;
    memcpy(&mp, &m.max_p_bits, sizeof(mp));
    out->max_p = mp;
    return SDM_OK;
}

}  // extern "C"
