// Regrouping gather + Monte-Carlo coalescence (paper Sec. 5.1.4).
//
// One launch per step handles every cell: it gathers the cell's
// super-droplets through the counting-sort permutation, orders them by id
// (so the stored layout, and with it every later floating-point sum, is
// independent of atomic arrival order), runs the sstp_coal substeps on the
// gathered copy and writes the cell contiguously into the other buffer.
//
// Per substep: the cell's n super-droplets with N > 0 are sorted by a
// Philox key (ties by id) and paired (0,1), (2,3), ...; pair k collides when
// its scaled probability, eq. (P_ij),
//     P = max(N_i, N_j) K(r_i, r_j) dt''/dV * n (n-1) / (2 floor(n/2)),
// exceeds the uniform number drawn for the pair's first member (with
// multiple coalescence on, floor(P) or floor(P) + 1 events: n_events).
//
// Cells of up to 64 super-droplets: one warp each, two per lane, a
// register bitonic sort through shuffles and per-warp shared memory for the
// attributes.  Larger cells (up to kBigCellCap): one block each, bitonic
// sort in shared memory, attributes in global memory.
#include "sdm_internal.cuh"

namespace sdm {

struct CoalParams {
    Grid g;
    int sstp, coal, kernel, mixed, multi, adapt;
    double golovin_b;
    uint64_t seed, step;
};

constexpr int kWarpsPerBlock = 4;

struct KeyRec {
    unsigned long long key, pk;  // sort key, then (id << 32 | slot)
};

__device__ __forceinline__ bool rec_less(const KeyRec &a, const KeyRec &b) {
    return a.key < b.key || (a.key == b.key && a.pk < b.pk);
}

__device__ __forceinline__ KeyRec shfl_rec(const KeyRec &r, int src) {
    KeyRec o;
    o.key = __shfl_sync(0xffffffffu, r.key, src);
    o.pk = __shfl_sync(0xffffffffu, r.pk, src);
    return o;
}

// bitonic sort of 32 R records, lane l holding positions R l .. R l + R - 1:
// exchanges across distance j < R stay in registers, longer ones go
// through shuffles with lane l ^ (j / R)
template <int R>
__device__ __forceinline__ void warp_sort(KeyRec (&v)[R], int lane) {
#pragma unroll
    for (int k = 2; k <= 32 * R; k <<= 1) {
#pragma unroll
        for (int j = k >> 1; j > 0; j >>= 1) {
            if (j < R) {
#pragma unroll
                for (int r = 0; r < R; ++r) {
                    const int rp = r ^ j;
                    if (rp > r) {
                        const bool up = ((R * lane + r) & k) == 0;
                        const bool sw = up ? rec_less(v[rp], v[r]) : rec_less(v[r], v[rp]);
                        if (sw) {
                            const KeyRec t = v[r];
                            v[r] = v[rp];
                            v[rp] = t;
                        }
                    }
                }
            } else {
                const int d = j / R;
                const int pl = lane ^ d;
                const bool lower = (lane & d) == 0;
#pragma unroll
                for (int r = 0; r < R; ++r) {
                    const bool up = ((R * lane + r) & k) == 0;
                    const KeyRec o = shfl_rec(v[r], pl);
                    const bool lt = rec_less(v[r], o);
                    if (up == lower) {
                        if (!lt) v[r] = o;
                    } else {
                        if (lt) v[r] = o;
                    }
                }
            }
        }
    }
}

// P_ij >= 0: its bit pattern orders like its value, so the statistics (the
// count of P > 1 and the largest P) take integer operations, not FP64 ones
constexpr unsigned long long kOneBits = 0x3FF0000000000000ull;  // 1.0

__device__ __forceinline__ unsigned long long p_bits(double P) {
    return (unsigned long long)__double_as_longlong(P);
}

// collection kernel: geometric (E = 1), Long (E = long_E) or Golovin; ra = sqrt(rw2a), rb =
// sqrt(rw2b), kept per super-droplet by the callers
template <bool EFF = true>
__device__ __forceinline__ double kernel_K(const CoalParams &p, double rw2a, double ra, double rw2b,
                                           double rb, double vta, double vtb) {
    if (p.kernel == SDM_KERNEL_GOLOVIN) {
        const double Va = 4.0 / 3.0 * phys::pi * rw2a * ra;
        const double Vb = 4.0 / 3.0 * phys::pi * rw2b * rb;
        return p.golovin_b * (Va + Vb);
    }
    const double dv = fabs(vta - vtb);
    const double K = phys::pi * (ra + rb) * (ra + rb) * dv;
    return EFF && p.kernel == SDM_KERNEL_LONG ? long_E(ra, rb) * K : K;
}

// Mixed-precision mode: terminal velocities, the kernel and P in FP32, a
// 24-bit uniform number and 32-bit shuffle keys (ties still broken by id);
// merged radii stay FP64 so that r^3 is conserved to FP64 rounding.
__device__ __forceinline__ double vt_of(const CoalParams &p, double rw2, double r, double nu, double cX) {
    return p.mixed ? (double)vterm_f((float)rw2, (float)nu, (float)cX) : vterm_r(rw2, r, nu, cX);
}

// EFF = false compiles the Long efficiency out (the variants that never see
// SDM_KERNEL_LONG)
template <bool EFF = true>
__device__ __forceinline__ double prob(const CoalParams &p, unsigned long long Nmax, double rwa, double ra,
                                       double rwb, double rb, double va, double vb, double dtpp, double scale) {
    if (p.mixed) {
        float K;
        if (p.kernel == SDM_KERNEL_GOLOVIN) {
            const float a = (float)rwa, b = (float)rwb;
            K = (float)p.golovin_b * (4.0f / 3.0f * (float)phys::pi) * (a * sqrtf(a) + b * sqrtf(b));
        } else {
            const float ra = sqrtf((float)rwa), rb = sqrtf((float)rwb);
            K = (float)phys::pi * (ra + rb) * (ra + rb) * fabsf((float)va - (float)vb);
            if (EFF && p.kernel == SDM_KERNEL_LONG) K = long_Ef(ra, rb) * K;
        }
        return (double)((float)Nmax * K * (float)dtpp / (float)p.g.dV * (float)scale);
    }
    const double K = kernel_K<EFF>(p, rwa, ra, rwb, rb, va, vb);
    return (double)Nmax * K * dtpp / p.g.dV * scale;
}

// mixed precision sorts on the 31 leading bits of the draw (ties fall back
// to id order), the key width the batched ensemble sorts on
__device__ __forceinline__ unsigned long long key_of(const CoalParams &p, uint64_t w0) {
    return p.mixed ? (w0 & 0xFFFFFFFE00000000ull) : w0;
}

// gamma collision events (gamma = 1 in the paper's scheme): the larger-N
// member L (the first on a tie) keeps its radii and loses gamma times the
// other's N; the other takes the merged droplet (r_w^3 and r_d^3 of gamma
// L-droplets added to its own, kappa weighted by r_d^3).  Returns the
// merged slot.
template <class Acc>
__device__ __forceinline__ int collide(Acc &A, int a, int b, unsigned long long gamma) {
    const int L = A.N(a) >= A.N(b) ? a : b;
    const int S = L == a ? b : a;
    A.setN(L, A.N(L) - gamma * A.N(S));
    const double g = (double)gamma;
    const double r3 = A.rw2(S) * A.r(S) + g * (A.rw2(L) * A.r(L));
    const double r = cbrt(r3);
    A.setrw2(S, r * r);
    const double dS = A.rd3(S), dL = g * A.rd3(L);
    const double m3 = dS + dL;
    if (m3 > 0.0) A.setkappa(S, (A.kappa(S) * dS + A.kappa(L) * dL) / m3);
    A.setrd3(S, m3);
    return S;
}

// Adaptive substeps (coal_adapt > 0; the paper plans substep control from
// P_ij, Sec. 5.1.4): from the cell's live count n, largest multiplicity,
// largest r_w^2 and terminal-velocity range at the start of the step, an
// upper bound of eq. P_ij over every pair the cell could form,
//   P_bound = N_max K_bound dt / dV * n (n-1) / (2 floor(n/2)),
// K_bound = pi (2 r_max)^2 (v_max - v_min) (geometric) or b 2 V_max
// (Golovin); the cell takes max(sstp_coal, ceil(P_bound)) substeps, at most
// coal_adapt.  Products only, so no contraction changes the rounding.
__device__ __forceinline__ int adaptive_sstp(const CoalParams &p, int n, unsigned long long Nmax, double rw2max,
                                             double vmax, double vmin) {
    if (p.adapt <= 0 || n < 2) return p.sstp;
    const double rmax = sqrt(rw2max);
    double K;
    if (p.kernel == SDM_KERNEL_GOLOVIN) {
        K = p.golovin_b * (2.0 * (4.0 / 3.0 * phys::pi * rw2max * rmax));
    } else {
        const double two_r = 2.0 * rmax;
        K = phys::pi * two_r * two_r * (vmax - vmin);
    }
    const double scale = pair_scale(n);
    const double Pb = (double)Nmax * K * p.g.dt / p.g.dV * scale;
    int s = p.sstp;
    if (Pb > (double)s) s = Pb >= (double)p.adapt ? p.adapt : (int)ceil(Pb);
    return s < p.sstp ? p.sstp : s;
}

__device__ __forceinline__ unsigned long long warp_max_u64(unsigned long long v) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        const unsigned long long w = __shfl_xor_sync(0xffffffffu, v, o);
        v = w > v ? w : v;
    }
    return v;
}

// ---------------------------------------------------------------- warp path
template <int CAP>
struct WarpSmem {
    unsigned long long N[CAP], acc[CAP];
    double rw2[CAP], r[CAP], rd3[CAP], kappa[CAP], vt[CAP];
    uint32_t uid[CAP];
};

template <int CAP>
struct SmemAcc {
    WarpSmem<CAP> *w;
    __device__ unsigned long long N(int i) const { return w->N[i]; }
    __device__ double rw2(int i) const { return w->rw2[i]; }
    __device__ double r(int i) const { return w->r[i]; }
    __device__ double rd3(int i) const { return w->rd3[i]; }
    __device__ double kappa(int i) const { return w->kappa[i]; }
    __device__ void setN(int i, unsigned long long v) { w->N[i] = v; }
    __device__ void setrw2(int i, double v) {
        w->rw2[i] = v;
        w->r[i] = sqrt(v);
    }
    __device__ void setrd3(int i, double v) { w->rd3[i] = v; }
    __device__ void setkappa(int i, double v) { w->kappa[i] = v; }
};

// cells of up to 32 R super-droplets, one warp each, R per lane.  EXT:
// multiple coalescence, adaptive substeps or the Long kernel on; the
// paper's scheme runs a copy without their code.
template <int R, bool EXT>
__global__ void __launch_bounds__(kWarpsPerBlock * 32)
    k_coal_warp(SdArrays src, SdArrays dst, const uint32_t *offset, const uint32_t *perm,
                const double *amb, CoalParams p, uint32_t *bigcells, DevStats *st) {
    constexpr int CAP = 32 * R;
    __shared__ WarpSmem<CAP> sm[kWarpsPerBlock];
    const int lane = threadIdx.x & 31, wib = threadIdx.x >> 5;
    const int c = blockIdx.x * kWarpsPerBlock + wib;
    if (c >= p.g.n_cells) return;
    WarpSmem<CAP> &W = sm[wib];
    const uint32_t beg = offset[c];
    const int n = (int)(offset[c + 1] - beg);
    if (n > CAP) {
        if (lane == 0) bigcells[atomicAdd(&st->n_big, 1u)] = (uint32_t)c;
        return;
    }
    // gather and order by id
    KeyRec v[R];
#pragma unroll
    for (int r = 0; r < R; ++r) {
        const int q = R * lane + r;
        v[r] = KeyRec{0, ~0ull};
        if (q < n) {
            const uint32_t pi = perm[beg + q];
            v[r].pk = ((unsigned long long)src.uid[pi] << 32) | pi;
        }
    }
    warp_sort<R>(v, lane);
    const double nu = amb[2 * c], cX = amb[2 * c + 1];
    const bool geo = p.kernel != SDM_KERNEL_GOLOVIN;  // kernels of terminal velocity
#pragma unroll
    for (int r = 0; r < R; ++r) {
        const int q = R * lane + r;
        if (q < n) {
            const uint32_t pi = (uint32_t)(v[r].pk & 0xffffffffu);
            const uint32_t id = (uint32_t)(v[r].pk >> 32);
            W.N[q] = src.N[pi];
            const double rw2 = src.rw2[pi];
            W.rw2[q] = rw2;
            W.r[q] = sqrt(rw2);
            W.rd3[q] = src.rd3[pi];
            W.kappa[q] = src.kappa[pi];
            W.uid[q] = id;
            W.vt[q] = geo ? vt_of(p, rw2, W.r[q], nu, cX) : 0.0;
            if (p.g.nx > 0) dst.x[beg + q] = src.x[pi];
            if (p.g.ny > 0) dst.y[beg + q] = src.y[pi];
            if (p.g.nz > 0) dst.z[beg + q] = src.z[pi];
            dst.uid[beg + q] = id;
        }
    }
    __syncwarp();
    unsigned long long n_pairs = 0, n_coll = 0, n_pgt1 = 0, max_pb = 0;
    int sstp = p.sstp;
    if (EXT && p.coal && p.adapt > 0) {
        int nl = 0;
        unsigned long long Nm = 0;
        double rm = 0.0, vmax = 0.0, vmin = INFINITY;
#pragma unroll
        for (int r = 0; r < R; ++r) {
            const int q = R * lane + r;
            if (q < n && W.N[q] > 0) {
                nl++;
                Nm = W.N[q] > Nm ? W.N[q] : Nm;
                rm = fmax(rm, W.rw2[q]);
                if (geo) {
                    vmax = fmax(vmax, W.vt[q]);
                    vmin = fmin(vmin, W.vt[q]);
                }
            }
        }
        nl = (int)__reduce_add_sync(0xffffffffu, (unsigned)nl);
        Nm = warp_max_u64(Nm);
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) {
            rm = fmax(rm, __shfl_xor_sync(0xffffffffu, rm, o));
            vmax = fmax(vmax, __shfl_xor_sync(0xffffffffu, vmax, o));
            vmin = fmin(vmin, __shfl_xor_sync(0xffffffffu, vmin, o));
        }
        sstp = adaptive_sstp(p, nl, Nm, rm, vmax, vmin);
    }
    if (p.coal && n >= 2) {
        SmemAcc<CAP> A{&W};
        const double dtpp = p.g.dt / sstp;
        for (int sub = 0; sub < sstp; ++sub) {
            int my_act = 0;
#pragma unroll
            for (int r = 0; r < R; ++r) {
                const int q = R * lane + r;
                v[r] = KeyRec{~0ull, ~0ull};
                if (q < n && W.N[q] > 0) {
                    const u64x4 w = philox4x64(W.uid[q], (uint64_t)sub, p.step, kStreamCoal, p.seed, 0);
                    W.acc[q] = w.v[1];
                    v[r] = KeyRec{key_of(p, w.v[0]), ((unsigned long long)W.uid[q] << 32) | (unsigned)q};
                    my_act++;
                }
            }
            const int m = __reduce_add_sync(0xffffffffu, (unsigned)my_act);
            __syncwarp();
            if (m < 2) continue;
            warp_sort<R>(v, lane);
            const double scale = pair_scale(m);
            // sorted positions R lane + r; pairs (2k, 2k + 1) are in one lane
            KeyRec pa[R >= 2 ? R / 2 : 1], pb[R >= 2 ? R / 2 : 1];
            if constexpr (R >= 2) {
#pragma unroll
                for (int r = 0; r < R; r += 2) {
                    pa[r / 2] = v[r];
                    pb[r / 2] = v[r + 1];
                }
            } else {  // one record per lane: the pair's second half is in lane + 1
                pa[0] = v[0];
                pb[0] = shfl_rec(v[0], lane ^ 1);
            }
#pragma unroll
            for (int h = 0; h < (R >= 2 ? R / 2 : 1); ++h) {
                const KeyRec ka = pa[h], kb = pb[h];
                const int pos = R >= 2 ? R * lane + 2 * h : lane;
                const bool mine = R >= 2 || (lane & 1) == 0;
                if (mine && pos + 1 < m) {
                    const int a = (int)(ka.pk & 0xffu), b = (int)(kb.pk & 0xffu);
                    const unsigned long long Na = W.N[a], Nb = W.N[b];
                    const unsigned long long Nmax = Na > Nb ? Na : Nb, Nmin = Na > Nb ? Nb : Na;
                    const double P = prob<EXT>(p, Nmax, W.rw2[a], W.r[a], W.rw2[b], W.r[b], W.vt[a], W.vt[b], dtpp,
                                          scale);
                    n_pairs++;
                    const unsigned long long pb = p_bits(P);
                    n_pgt1 += pb > kOneBits;
                    max_pb = pb > max_pb ? pb : max_pb;
                    const unsigned long long gam =
                        n_events(P, W.acc[a], Nmax, Nmin, EXT ? p.multi : 0, p.mixed);
                    if (gam) {
                        const int S = collide(A, a, b, gam);
                        if (geo) W.vt[S] = vt_of(p, W.rw2[S], W.r[S], nu, cX);
                        n_coll++;
                    }
                }
            }
            __syncwarp();
        }
    }
    unsigned zeros = 0;
#pragma unroll
    for (int r = 0; r < R; ++r) {
        const int q = R * lane + r;
        if (q < n) {
            dst.N[beg + q] = W.N[q];
            dst.rw2[beg + q] = W.rw2[q];
            dst.rd3[beg + q] = W.rd3[q];
            dst.kappa[beg + q] = W.kappa[q];
            zeros += W.N[q] == 0;
        }
    }
    zeros = __reduce_add_sync(0xffffffffu, zeros);
    const unsigned np = __reduce_add_sync(0xffffffffu, (unsigned)n_pairs);
    const unsigned nc = __reduce_add_sync(0xffffffffu, (unsigned)n_coll);
    const unsigned ng = __reduce_add_sync(0xffffffffu, (unsigned)n_pgt1);
    max_pb = warp_max_u64(max_pb);
    if (lane == 0) {
        if (p.coal) atomicAdd(&st->n_coal_substeps, (unsigned long long)sstp);
        if (zeros) atomicAdd(&st->n_zero, (unsigned long long)zeros);
        if (np) atomicAdd(&st->n_pairs, (unsigned long long)np);
        if (nc) atomicAdd(&st->n_coll, (unsigned long long)nc);
        if (ng) atomicAdd(&st->n_pgt1, (unsigned long long)ng);
        if (max_pb) atomicMax(&st->max_p_bits, max_pb);
    }
}

// ---------------------------------------------------------------- block path
struct GlobalAcc {
    SdArrays s;
    uint32_t beg;
    __device__ unsigned long long N(int i) const { return s.N[beg + i]; }
    __device__ double rw2(int i) const { return s.rw2[beg + i]; }
    __device__ double r(int i) const { return sqrt(s.rw2[beg + i]); }
    __device__ double rd3(int i) const { return s.rd3[beg + i]; }
    __device__ double kappa(int i) const { return s.kappa[beg + i]; }
    __device__ void setN(int i, unsigned long long v) { s.N[beg + i] = v; }
    __device__ void setrw2(int i, double v) { s.rw2[beg + i] = v; }
    __device__ void setrd3(int i, double v) { s.rd3[beg + i] = v; }
    __device__ void setkappa(int i, double v) { s.kappa[beg + i] = v; }
};

constexpr int kBigBlock = 1024;

__device__ void block_sort(unsigned long long *key, unsigned long long *pk, int npow2) {
    for (int k = 2; k <= npow2; k <<= 1) {
        for (int j = k >> 1; j > 0; j >>= 1) {
            for (int i = threadIdx.x; i < npow2; i += blockDim.x) {
                const int ixj = i ^ j;
                if (ixj > i) {
                    const bool up = (i & k) == 0;
                    const unsigned long long ka = key[i], kb = key[ixj], pa = pk[i], pb = pk[ixj];
                    const bool a_gt = ka > kb || (ka == kb && pa > pb);
                    if (a_gt == up) {
                        key[i] = kb;
                        key[ixj] = ka;
                        pk[i] = pb;
                        pk[ixj] = pa;
                    }
                }
            }
            __syncthreads();
        }
    }
}

// huge (may be null): scratch for cells above kBigCellCap, three arrays of
// 2 n_sd records (a cell at twice its offset, so that the power-of-two
// padding of one cell never reaches the next); those cells take the same
// steps on global memory, slower but with the same results
__global__ void __launch_bounds__(kBigBlock)
    k_coal_block(SdArrays src, SdArrays dst, const uint32_t *offset, const uint32_t *perm,
                 const double *amb, CoalParams p, const uint32_t *bigcells, DevStats *st,
                 unsigned long long *huge, int64_t n_sd) {
    extern __shared__ unsigned long long smem[];
    __shared__ int s_m;
    __shared__ unsigned long long s_cnt[4];
    __shared__ unsigned long long s_maxp;
    __shared__ unsigned long long s_Nm[32];
    __shared__ double s_rm[32], s_vmax[32], s_vmin[32];
    __shared__ int s_n[32], s_sstp;
    const unsigned nbig = st->n_big;
    for (unsigned bi = blockIdx.x; bi < nbig; bi += gridDim.x) {
        const int c = (int)bigcells[bi];
        const uint32_t beg = offset[c];
        const int n = (int)(offset[c + 1] - beg);
        unsigned long long *skey = smem, *spk = smem + kBigCellCap, *sacc = smem + 2 * kBigCellCap;
        if (n > kBigCellCap) {
            if (!huge) {
                if (threadIdx.x == 0) atomicOr(&st->flags, kFlagBigCell);
                continue;
            }
            skey = huge + 2 * (int64_t)beg;
            spk = huge + 2 * n_sd + 2 * (int64_t)beg;
            sacc = huge + 4 * n_sd + 2 * (int64_t)beg;
        }
        int npow2 = 1;
        while (npow2 < n) npow2 <<= 1;
        for (int t = threadIdx.x; t < npow2; t += blockDim.x) {
            skey[t] = 0;
            if (t < n) {
                const uint32_t pi = perm[beg + t];
                spk[t] = ((unsigned long long)src.uid[pi] << 32) | pi;
            } else {
                spk[t] = ~0ull;
            }
        }
        __syncthreads();
        // already in id order (a one-cell domain keeps its storage order
        // through the counting sort): no sort
        bool ordered = true;
        for (int t = threadIdx.x; t + 1 < n; t += blockDim.x) ordered &= spk[t] < spk[t + 1];
        if (!__syncthreads_and(ordered)) block_sort(skey, spk, npow2);
        for (int t = threadIdx.x; t < n; t += blockDim.x) {
            const uint32_t pi = (uint32_t)(spk[t] & 0xffffffffu);
            const uint32_t o = beg + t;
            dst.N[o] = src.N[pi];
            dst.rw2[o] = src.rw2[pi];
            dst.rd3[o] = src.rd3[pi];
            dst.kappa[o] = src.kappa[pi];
            if (p.g.nx > 0) dst.x[o] = src.x[pi];
            if (p.g.ny > 0) dst.y[o] = src.y[pi];
            if (p.g.nz > 0) dst.z[o] = src.z[pi];
            dst.uid[o] = (uint32_t)(spk[t] >> 32);
        }
        if (threadIdx.x < 4) s_cnt[threadIdx.x] = 0;
        if (threadIdx.x == 0) s_maxp = 0;
        __syncthreads();
        const double nu = amb[2 * c], cX = amb[2 * c + 1];
        const bool geo = p.kernel != SDM_KERNEL_GOLOVIN;  // kernels of terminal velocity
        GlobalAcc A{dst, beg};
        if (threadIdx.x == 0) s_sstp = p.sstp;
        if (p.coal && p.adapt > 0) {  // adaptive_sstp from a block reduction
            int nl = 0;
            unsigned long long Nm = 0;
            double rm = 0.0, vmax = 0.0, vmin = INFINITY;
            for (int t = threadIdx.x; t < n; t += blockDim.x) {
                const unsigned long long Nt = dst.N[beg + t];
                if (Nt == 0) continue;
                const double rw2 = dst.rw2[beg + t];
                nl++;
                Nm = Nt > Nm ? Nt : Nm;
                rm = fmax(rm, rw2);
                if (geo) {
                    const double v = vt_of(p, rw2, sqrt(rw2), nu, cX);
                    vmax = fmax(vmax, v);
                    vmin = fmin(vmin, v);
                }
            }
            nl = (int)__reduce_add_sync(0xffffffffu, (unsigned)nl);
            Nm = warp_max_u64(Nm);
            for (int o = 16; o > 0; o >>= 1) {
                rm = fmax(rm, __shfl_xor_sync(0xffffffffu, rm, o));
                vmax = fmax(vmax, __shfl_xor_sync(0xffffffffu, vmax, o));
                vmin = fmin(vmin, __shfl_xor_sync(0xffffffffu, vmin, o));
            }
            const int wid = threadIdx.x >> 5, nw = blockDim.x >> 5;
            if ((threadIdx.x & 31) == 0) {
                s_n[wid] = nl;
                s_Nm[wid] = Nm;
                s_rm[wid] = rm;
                s_vmax[wid] = vmax;
                s_vmin[wid] = vmin;
            }
            __syncthreads();
            if (threadIdx.x == 0) {
                for (int k = 1; k < nw; ++k) {
                    nl += s_n[k];
                    Nm = s_Nm[k] > Nm ? s_Nm[k] : Nm;
                    rm = fmax(rm, s_rm[k]);
                    vmax = fmax(vmax, s_vmax[k]);
                    vmin = fmin(vmin, s_vmin[k]);
                }
                s_sstp = adaptive_sstp(p, nl, Nm, rm, vmax, vmin);
            }
        }
        __syncthreads();
        const int sstp = s_sstp;
        if (threadIdx.x == 0 && p.coal) atomicAdd(&st->n_coal_substeps, (unsigned long long)sstp);
        if (p.coal && n >= 2) {
            const double dtpp = p.g.dt / sstp;
            for (int sub = 0; sub < sstp; ++sub) {
                if (threadIdx.x == 0) s_m = 0;
                __syncthreads();
                int my_m = 0;
                for (int t = threadIdx.x; t < npow2; t += blockDim.x) {
                    if (t < n && dst.N[beg + t] > 0) {
                        const uint32_t id = dst.uid[beg + t];
                        const u64x4 w = philox4x64(id, (uint64_t)sub, p.step, kStreamCoal, p.seed, 0);
                        skey[t] = key_of(p, w.v[0]);
                        sacc[t] = w.v[1];
                        spk[t] = ((unsigned long long)id << 32) | (unsigned)t;
                        my_m++;
                    } else {
                        skey[t] = ~0ull;
                        spk[t] = ~0ull;
                    }
                }
                atomicAdd(&s_m, my_m);
                __syncthreads();
                const int m = s_m;
                if (m < 2) {
                    __syncthreads();
                    continue;
                }
                block_sort(skey, spk, npow2);
                const double scale = pair_scale(m);
                unsigned long long np = 0, nc = 0, ng = 0, mpb = 0;
                for (int k = threadIdx.x; k < m / 2; k += blockDim.x) {
                    const int a = (int)(spk[2 * k] & 0xffffffffu), b = (int)(spk[2 * k + 1] & 0xffffffffu);
                    const double rwa = A.rw2(a), rwb = A.rw2(b), ra = sqrt(rwa), rb = sqrt(rwb);
                    const unsigned long long Na = A.N(a), Nb = A.N(b);
                    const unsigned long long Nmax = Na > Nb ? Na : Nb, Nmin = Na > Nb ? Nb : Na;
                    const double P = prob(p, Nmax, rwa, ra, rwb, rb, geo ? vt_of(p, rwa, ra, nu, cX) : 0.0,
                                          geo ? vt_of(p, rwb, rb, nu, cX) : 0.0, dtpp, scale);
                    np++;
                    const unsigned long long pb = p_bits(P);
                    ng += pb > kOneBits;
                    mpb = pb > mpb ? pb : mpb;
                    const unsigned long long gam = n_events(P, sacc[a], Nmax, Nmin, p.multi, p.mixed);
                    if (gam) {
                        collide(A, a, b, gam);
                        nc++;
                    }
                }
                if (np) atomicAdd(&s_cnt[0], np);
                if (nc) atomicAdd(&s_cnt[1], nc);
                if (ng) atomicAdd(&s_cnt[2], ng);
                if (mpb) atomicMax(&s_maxp, mpb);
                __syncthreads();
            }
        }
        unsigned z = 0;
        for (int t = threadIdx.x; t < n; t += blockDim.x) z += dst.N[beg + t] == 0;
        if (z) atomicAdd(&s_cnt[3], (unsigned long long)z);
        __syncthreads();
        if (threadIdx.x == 0) {
            if (s_cnt[0]) atomicAdd(&st->n_pairs, s_cnt[0]);
            if (s_cnt[1]) atomicAdd(&st->n_coll, s_cnt[1]);
            if (s_cnt[2]) atomicAdd(&st->n_pgt1, s_cnt[2]);
            if (s_cnt[3]) atomicAdd(&st->n_zero, s_cnt[3]);
            if (s_maxp) atomicMax(&st->max_p_bits, s_maxp);
        }
        __syncthreads();
    }
}

cudaError_t launch_coalesce(sdm_ctx *c, const sdm_opts &o, bool coal) {
    CoalParams p;
    p.g = c->grid;
    p.sstp = o.sstp_coal;
    p.coal = coal ? 1 : 0;
    p.kernel = c->oi.kernel;
    p.mixed = c->oi.precision == SDM_PRECISION_MIXED;
    p.multi = o.coal_multi ? 1 : 0;
    p.adapt = o.coal_adapt;
    p.golovin_b = c->oi.golovin_b;
    p.seed = c->oi.seed;
    p.step = c->step;
    SdArrays src = c->buf[c->cur], dst = c->buf[c->cur ^ 1];
    cudaError_t e = cudaMemsetAsync(&c->dstats->n_big, 0, sizeof(unsigned), c->stream);
    if (e == cudaSuccess) e = cudaMemsetAsync(&c->dstats->n_zero, 0, sizeof(unsigned long long), c->stream);
    if (e != cudaSuccess) return e;
    const int nb = (c->grid.n_cells + kWarpsPerBlock - 1) / kWarpsPerBlock;
    // records per lane: cells hold sd_conc on average and spread around it
    // as super-droplets move, so the warp path covers twice the mean
    const int per_cell = c->G * c->oi.sd_conc;
    const bool ext = p.multi || p.adapt > 0 || p.kernel == SDM_KERNEL_LONG;
    auto launch = [&](auto kern) {
        kern<<<nb, kWarpsPerBlock * 32, 0, c->stream>>>(src, dst, c->offset, c->perm, c->amb, p, c->bigcells,
                                                        c->dstats);
    };
    if (per_cell <= 16) ext ? launch(k_coal_warp<1, true>) : launch(k_coal_warp<1, false>);
    else if (per_cell <= 32) ext ? launch(k_coal_warp<2, true>) : launch(k_coal_warp<2, false>);
    else ext ? launch(k_coal_warp<4, true>) : launch(k_coal_warp<4, false>);
    e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    const size_t smem = sizeof(unsigned long long) * 3 * kBigCellCap;
    static std::atomic<unsigned long long> attr_done{0};
    e = smem_attr_once(k_coal_block, (int)smem, attr_done);
    if (e != cudaSuccess) return e;
    int nsm = 0;
    cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, c->device);
    int blocks = nsm > 0 ? nsm : 152;
    if (blocks > c->grid.n_cells) blocks = c->grid.n_cells;
    k_coal_block<<<blocks, kBigBlock, smem, c->stream>>>(src, dst, c->offset, c->perm, c->amb, p,
                                                         c->bigcells, c->dstats, c->huge, c->n_sd);
    return cudaGetLastError();
}

}  // namespace sdm
