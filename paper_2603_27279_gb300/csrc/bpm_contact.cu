// Hertz-Mindlin contact between non-bonded particles (Methods, "Contact":
// the paper uses a Hertz-Mindlin granular model between particles that are
// not bonded neighbours; the force law below is the textbook one, stated in
// include/bpm.h).
//
// Per force evaluation:
//   1. cell list: each particle's cell (side = largest contact distance)
//      is hashed into H buckets; bucket counts, their exclusive prefix sum,
//      a scatter of particle indices and a per-bucket insertion sort give
//      the particles of every bucket in ascending index order, so the
//      neighbour visits (and the force sums) are the same on every run;
//   2. contact kernel, one thread per particle i, in two phases.  Phase A
//      (FP32 and integer work only): the 27 neighbouring cells' buckets
//      (each bucket once), the bonded-neighbour exclusion and an FP32
//      overlap filter whose margin bounds the FP32 rounding of the distance,
//      collecting candidates in a per-thread list.  Phase B (FP64): the
//      exact overlap test and the pair law for each candidate, the warp's
//      lanes stepping through their lists together, and the tangential
//      history of (i, j) read from the reference level and written to the
//      output level.  GB300 issues FP64 at 1/64 of the FP32 rate, so the
//      filter keeps FP64 work to the real contacts.  Both particles of a
//      pair evaluate it with sign-symmetric arithmetic, so f_j = -f_i holds
//      exactly and no atomics are needed.
#include "bpm_devmath.cuh"
#include "bpm_internal.h"

namespace bpm {

namespace {

constexpr int SCAN_T = 1024;          // threads of a scan block
constexpr int SCAN_CHUNK = 2 * SCAN_T;  // entries per scan block
constexpr int CT_T = 128;             // threads of the contact kernel

__device__ __forceinline__ int64_t cell_of(double x, double inv) {
    double c = floor(x * inv);
    c = fmin(fmax(c, -1e15), 1e15);
    return (int64_t)c;
}

__device__ __forceinline__ uint32_t bucket_of(int64_t cx, int64_t cy, int64_t cz, uint32_t mask) {
    uint64_t h = (uint64_t)cx * 0x9E3779B185EBCA87ull;
    h ^= (uint64_t)cy * 0xC2B2AE3D27D4EB4Full;
    h ^= (uint64_t)cz * 0x165667B19E3779F9ull;
    h ^= h >> 31;
    h *= 0xD6E8FEB86659FD93ull;
    h ^= h >> 32;
    return (uint32_t)h & mask;
}

__global__ void __launch_bounds__(256) k_ct_key_count(Sys s, Contact c) {
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= s.n) return;
    const int64_t n = s.n;
    const uint32_t b = bucket_of(cell_of(s.x[i], c.inv_cell), cell_of(s.x[n + i], c.inv_cell),
                                 cell_of(s.x[2 * n + i], c.inv_cell), c.H - 1);
    c.key[i] = (int)b;
    atomicAdd(c.count + b, 1);
    c.xf[i] = __double2float_rn(s.x[i]);
    c.xf[n + i] = __double2float_rn(s.x[n + i]);
    c.xf[2 * n + i] = __double2float_rn(s.x[2 * n + i]);
}

// exclusive scan of the pair (a0, a1) of every thread of a 1024-thread block
__device__ __forceinline__ void block_scan2(int a0, int a1, int& e0, int& e1, int& total) {
    __shared__ int warp_tot[SCAN_T / 32];
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    const int v = a0 + a1;
    int x = v;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        const int y = __shfl_up_sync(0xffffffffu, x, o);
        if (lane >= o) x += y;
    }
    if (lane == 31) warp_tot[w] = x;
    __syncthreads();
    if (w == 0) {
        int t = warp_tot[lane];
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const int y = __shfl_up_sync(0xffffffffu, t, o);
            if (lane >= o) t += y;
        }
        warp_tot[lane] = t;  // inclusive over warps
    }
    __syncthreads();
    const int before = (w > 0 ? warp_tot[w - 1] : 0) + x - v;
    e0 = before;
    e1 = before + a0;
    total = warp_tot[SCAN_T / 32 - 1];
}

// out[k] = sum of in[0..k) within each chunk of SCAN_CHUNK; bsum[b] = chunk total
__global__ void __launch_bounds__(SCAN_T) k_scan_local(const int* in, int* out, int* bsum, uint32_t H) {
    const uint32_t k0 = blockIdx.x * SCAN_CHUNK + 2 * threadIdx.x;
    const int a0 = k0 < H ? in[k0] : 0;
    const int a1 = k0 + 1 < H ? in[k0 + 1] : 0;
    int e0, e1, tot;
    block_scan2(a0, a1, e0, e1, tot);
    if (k0 < H) out[k0] = e0;
    if (k0 + 1 < H) out[k0 + 1] = e1;
    if (threadIdx.x == 0) bsum[blockIdx.x] = tot;
}

// exclusive scan of the nb <= SCAN_CHUNK chunk totals in place; *total = sum
__global__ void __launch_bounds__(SCAN_T) k_scan_top(int* bsum, int nb, int* total) {
    const int k0 = 2 * threadIdx.x;
    const int a0 = k0 < nb ? bsum[k0] : 0;
    const int a1 = k0 + 1 < nb ? bsum[k0 + 1] : 0;
    int e0, e1, tot;
    block_scan2(a0, a1, e0, e1, tot);
    if (k0 < nb) bsum[k0] = e0;
    if (k0 + 1 < nb) bsum[k0 + 1] = e1;
    if (threadIdx.x == 0) *total = tot;
}

__global__ void __launch_bounds__(SCAN_T) k_scan_add(int* out, const int* bsum, uint32_t H) {
    const int add = bsum[blockIdx.x];
    const uint32_t k0 = blockIdx.x * SCAN_CHUNK + 2 * threadIdx.x;
    if (k0 < H) out[k0] += add;
    if (k0 + 1 < H) out[k0 + 1] += add;
}

// count[] returns to zero as the slots of each bucket are handed out
__global__ void __launch_bounds__(256) k_ct_scatter(Sys s, Contact c) {
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= s.n) return;
    const int b = c.key[i];
    const int slot = atomicSub(c.count + b, 1) - 1;
    c.order[c.start[b] + slot] = (int)i;
}

__global__ void __launch_bounds__(256) k_ct_sort(Contact c) {
    const uint32_t b = blockIdx.x * blockDim.x + threadIdx.x;
    if (b >= c.H) return;
    const int lo = c.start[b], hi = c.start[b + 1];
    for (int p = lo + 1; p < hi; ++p) {
        const int v = c.order[p];
        int q = p - 1;
        while (q >= lo && c.order[q] > v) {
            c.order[q + 1] = c.order[q];
            --q;
        }
        c.order[q + 1] = v;
    }
}

// R_i w_i + R_j w_j without fused multiply-adds: the same bits for (i, j)
// and (j, i)
__device__ __forceinline__ d3 wsum_sym(d3 wi, double Ri, d3 wj, double Rj) {
    return mk3(__dadd_rn(__dmul_rn(wi.x, Ri), __dmul_rn(wj.x, Rj)),
               __dadd_rn(__dmul_rn(wi.y, Ri), __dmul_rn(wj.y, Rj)),
               __dadd_rn(__dmul_rn(wi.z, Ri), __dmul_rn(wj.z, Rj)));
}

constexpr int CT_MAXC = 64;  // candidates kept per particle (= largest cap)

__global__ void __launch_bounds__(CT_T) k_contact(Sys s, Contact c) {
    const int64_t n = s.n;
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    // levels: a step's evaluation reads the current level and writes the
    // previous one's buffers; a stand-alone one reads the previous level and
    // fills in the current level when it is empty
    const int cur = *s.hist_gen & 1, prv = cur ^ 1;
    const bool step = s.count_step != 0;
    const int ref = step ? cur : prv;
    const int out = step ? prv : (s.ct_valid[cur] ? -1 : cur);
    const int nref = s.ct_valid[ref] ? c.ncont[(size_t)ref * n + i] : 0;
    const size_t capn = (size_t)c.cap * n;
    const int* pref = c.partner + (size_t)ref * capn;
    const double* xref = c.xi + (size_t)ref * 3 * capn;
    int* pout = c.partner + (size_t)(out < 0 ? 0 : out) * capn;
    double* xout = c.xi + (size_t)(out < 0 ? 0 : out) * 3 * capn;
    const int rod_i = s.rod_of[i];

    // ---- phase A: candidates (FP32 filter)
    int cand[CT_MAXC];
    int ncand = 0;
    bool over = false;
    {
        const float xfi = c.xf[i], yfi = c.xf[n + i], zfi = c.xf[2 * n + i];
        const float rfi = c.radf[i];
        const float mi = fmaxf(fabsf(xfi), fmaxf(fabsf(yfi), fabsf(zfi)));
        const int64_t cx = cell_of(s.x[i], c.inv_cell), cy = cell_of(s.x[n + i], c.inv_cell),
                      cz = cell_of(s.x[2 * n + i], c.inv_cell);
        const uint32_t mask = c.H - 1;
        uint32_t seen[27];
        int ns = 0;
        for (int dz = -1; dz <= 1; ++dz)
            for (int dy = -1; dy <= 1; ++dy)
                for (int dx = -1; dx <= 1; ++dx) {
                    const uint32_t b = bucket_of(cx + dx, cy + dy, cz + dz, mask);
                    bool dup = false;
                    for (int k = 0; k < ns; ++k) dup |= seen[k] == b;
                    if (dup) continue;
                    seen[ns++] = b;
                    const int hi = c.start[b + 1];
                    for (int p = c.start[b]; p < hi; ++p) {
                        const int j = c.order[p];
                        if (j == i) continue;
                        const int64_t dij = j > i ? j - i : i - j;
                        if (dij <= c.exclude && s.rod_of[j] == rod_i) continue;
                        const float xfj = c.xf[j], yfj = c.xf[n + j], zfj = c.xf[2 * n + j];
                        const float ddx = xfi - xfj, ddy = yfi - yfj, ddz = zfi - zfj;
                        const float d2 = fmaf(ddx, ddx, fmaf(ddy, ddy, ddz * ddz));
                        // the FP32 distance is within 2^-21 (|x|max + R_i + R_j)
                        // of the exact one; the margin is 4 times that
                        const float rs = rfi + c.radf[j];
                        const float mj = fmaxf(fabsf(xfj), fmaxf(fabsf(yfj), fabsf(zfj)));
                        const float lim = fmaf(0x1p-19f, fmaxf(mi, mj) + rs, rs);
                        if (d2 < lim * lim) {
                            if (ncand < CT_MAXC)
                                cand[ncand++] = j;
                            else
                                over = true;
                        }
                    }
                }
    }

    // ---- phase B: exact test and pair law (FP64)
    const d3 xi = mk3(s.x[i], s.x[n + i], s.x[2 * n + i]);
    const d3 vi = mk3(s.v[i], s.v[n + i], s.v[2 * n + i]);
    const d3 wi = mk3(s.w[i], s.w[n + i], s.w[2 * n + i]);
    const double Ri = c.radius[i];
    d3 F = mk3(0, 0, 0), T = mk3(0, 0, 0);
    int nc = 0;
    for (int k = 0; k < ncand; ++k) {
        const int j = cand[k];
        const d3 d = xi - mk3(s.x[j], s.x[n + j], s.x[2 * n + j]);
        const double Rj = c.radius[j];
        const double Rs = Ri + Rj;
        const double dist2 = dot(d, d);
        if (!(dist2 < Rs * Rs) || !(dist2 > 0.0)) continue;
        const double rinv = rsqrt_nr(dist2);
        const double delta = Rs - dist2 * rinv;
        if (!(delta > 0.0)) continue;
        const d3 nv = d * rinv;
        const double tA = Ri * Rj * rcp_nr(Rs) * delta;  // R* delta
        const double a = tA * rsqrt_nr(tA);              // contact radius
        const double Fh = (4.0 / 3.0) * c.E_star * a * delta;  // Hertz
        const d3 vj = mk3(s.v[j], s.v[n + j], s.v[2 * n + j]);
        const d3 wj = mk3(s.w[j], s.w[n + j], s.w[2 * n + j]);
        const d3 vrel = (vi - vj) - cross(wsum_sym(wi, Ri, wj, Rj), nv);
        const double vn = dot(vrel, nv);
        const d3 vt = vrel - nv * vn;
        // tangential history of (i, j), carried into the current plane
        d3 xo = mk3(0, 0, 0);
        for (int r = 0; r < nref; ++r)
            if (pref[(size_t)r * n + i] == j) {
                const size_t o = (size_t)r * n + i;
                xo = mk3(xref[o], xref[capn + o], xref[2 * capn + o]);
                const d3 xp = xo - nv * dot(xo, nv);
                const double lo2 = dot(xo, xo), lp2 = dot(xp, xp);
                xo = lp2 > 0.0 ? xp * (lo2 * rsqrt_nr(lo2) * rsqrt_nr(lp2)) : xp;
                break;
            }
        d3 xin = xo + vt * s.dt;
        const double kt = 8.0 * c.G_star * a;  // Mindlin
        d3 Ft = xin * (-kt) - vt * c.gamma_t;
        const double fmax = c.mu * Fh;
        const double ft2 = dot(Ft, Ft);
        if (ft2 > fmax * fmax) {
            Ft = Ft * (fmax * rsqrt_nr(ft2));
            xin = (Ft + vt * c.gamma_t) * (-rcp_nr(kt));
        }
        F = F + nv * (Fh - c.gamma_n * vn) + Ft;
        T = T + cross(nv * (-Ri), Ft);
        if (out >= 0) {
            if (nc < c.cap) {
                const size_t o = (size_t)nc * n + i;
                pout[o] = j;
                xout[o] = xin.x;
                xout[capn + o] = xin.y;
                xout[2 * capn + o] = xin.z;
                ++nc;
            } else {
                over = true;
            }
        } else if (++nc > c.cap) {
            over = true;
        }
    }
    if (out >= 0) c.ncont[(size_t)out * n + i] = nc;
    if (over) atomicExch(c.overflow, 1);
    s.f[i] += F.x;
    s.f[n + i] += F.y;
    s.f[2 * n + i] += F.z;
    s.t[i] += T.x;
    s.t[n + i] += T.y;
    s.t[2 * n + i] += T.z;
}

}  // namespace

int contact_scan_blocks(uint32_t H) { return (int)((H + SCAN_CHUNK - 1) / SCAN_CHUNK); }

cudaError_t launch_contact(const Sys& s, const Contact& c, cudaStream_t st) {
    if (s.n == 0) return cudaSuccess;
    const unsigned gn = (unsigned)((s.n + 255) / 256);
    const int nb = contact_scan_blocks(c.H);
    if (nb > SCAN_CHUNK) return cudaErrorInvalidValue;  // H above 2^22: rejected at create
    k_ct_key_count<<<gn, 256, 0, st>>>(s, c);
    k_scan_local<<<nb, SCAN_T, 0, st>>>(c.count, c.start, c.block_sums, c.H);
    k_scan_top<<<1, SCAN_T, 0, st>>>(c.block_sums, nb, c.start + c.H);
    k_scan_add<<<nb, SCAN_T, 0, st>>>(c.start, c.block_sums, c.H);
    k_ct_scatter<<<gn, 256, 0, st>>>(s, c);
    k_ct_sort<<<(c.H + 255) / 256, 256, 0, st>>>(c);
    k_contact<<<(unsigned)((s.n + CT_T - 1) / CT_T), CT_T, 0, st>>>(s, c);
    return cudaGetLastError();
}

}  // namespace bpm
