// sort.cu -- orientation + spaxel keys (Sec. 3: the galaxy is rotated into the
// field of view and each particle is assigned to an IFU spaxel) and the
// deterministic stable sort of particles by spaxel that replaces global
// atomics in the per-spaxel sum of spectra.
#include "common.cuh"
#include "kernels.h"

namespace rubix {

// ----------------------------------------------------------------------------
// K1: orientation + spaxel key. Reading: with the orientation matrix R built
// on the host (R = Rz(position angle) Rx(inclination) Rz(azimuth), its
// elements rounded as the ABI header states, no contraction),
// x' = (R00 x + R01 y) + R02 z, y' likewise, v_los = (R20 vx + R21 vy) + R22 vz;
// x_lo = (-0.5 nx) size; u = (x' - x_lo) * (1/size) with every FP64 op
// rounded once, so the integer key is bit-identical to a host evaluation of
// the same expression. On this GPU the FP64 pipe runs at 1/64 of the FP32
// rate, so u is first estimated in FP32 with a bound on its error; only
// particles whose estimate lies within that bound of a spaxel edge (about
// 0.1 %) evaluate the FP64 expression (key_coord_fp32). v_los, which decides
// no integer, is evaluated in FP32. Pre-projected input takes (x', y',
// v_los) as given. With a row window the key counts rows from its first row and
// particles of other rows are dropped like those outside the field.
// With age bands the sort key appends the particle's band (an internal
// partition of the SSP grid used by the deposit) below the spaxel index.
// ----------------------------------------------------------------------------
// FP32 estimate est of one key coordinate (x' or y' in spaxel units) and a
// bound err >= |est - u| on its distance from the FP64 value u of the
// reading. The FP32 path (R and the inputs rounded to FP32, products and
// sums by FMA) carries at most ~8 FP32 roundings of the terms' magnitudes,
// |est - u| <= 2^-21 (|R0 X| + |R1 Y| + |R2 Z| + |x_lo|) / size; err takes
// 2^-19 of that sum plus |est| (the rounding of est +- err itself) and 1.
// When no integer lies within err of est, floor(u) = floor(est) and the key
// coordinate is decided in FP32; otherwise (a fraction ~4 err of particles,
// about 0.1 % for the fields here) it is recomputed in FP64 exactly as the
// reading states. Returns false if undecided; else k = floor(u), possibly
// outside [0, n).
__device__ __forceinline__ bool key_coord_fp32(float est, float mag, int& k) {
    const float err = 0x1p-19f * (mag + fabsf(est) + 1.f);
    const float lo = floorf(est - err), hi = floorf(est + err);
    if (lo != hi) return false;
    // |est| beyond the int range: outside any field
    k = (fabsf(lo) < 1e9f) ? (int)lo : -1;
    return true;
}

__global__ void k_assign(AssignParams P) {
    const long long n = P.n;
    // the orientation and field constants in FP32 for the fast path
    float Rf[9];
#pragma unroll
    for (int i = 0; i < 9; ++i) Rf[i] = (float)P.R[i];
    const float xlo_f = (float)P.x_lo, ylo_f = (float)P.y_lo, inv_f = (float)P.inv_size;
    for (long long p = blockIdx.x * (long long)blockDim.x + threadIdx.x; p < n;
         p += (long long)gridDim.x * blockDim.x) {
        float X = 0.f, Y = 0.f, Z = 0.f, v = 0.f;
        float xe, ye, mx, my;  // FP32 key coordinates and their magnitude sums
        if (P.preprojected) {
            X = P.x[p];
            Y = P.y[p];
            v = P.v_los ? P.v_los[p] : 0.f;
            if (P.dv_dang) P.dv_dang[p] = make_float2(0.f, 0.f);
            xe = (X - xlo_f) * inv_f;
            ye = (Y - ylo_f) * inv_f;
            mx = (fabsf(X) + fabsf(xlo_f)) * inv_f;
            my = (fabsf(Y) + fabsf(ylo_f)) * inv_f;
        } else {
            X = P.x[p];
            Y = P.y[p];
            Z = P.z[p];
            const float xp = fmaf(Rf[2], Z, fmaf(Rf[1], Y, Rf[0] * X));
            const float yp = fmaf(Rf[5], Z, fmaf(Rf[4], Y, Rf[3] * X));
            xe = (xp - xlo_f) * inv_f;
            ye = (yp - ylo_f) * inv_f;
            mx = (fabsf(Rf[0] * X) + fabsf(Rf[1] * Y) + fabsf(Rf[2] * Z) + fabsf(xlo_f)) * inv_f;
            my = (fabsf(Rf[3] * X) + fabsf(Rf[4] * Y) + fabsf(Rf[5] * Z) + fabsf(ylo_f)) * inv_f;
            // the line-of-sight velocity feeds the Doppler factor (FP32 FMAs;
            // it decides no integer)
            if (P.vy) {
                const float VX = P.vx ? P.vx[p] : 0.f, VY = P.vy[p], VZ = P.vz[p];
                v = fmaf(Rf[8], VZ, fmaf(Rf[7], VY, Rf[6] * VX));
                if (P.dv_dang)
                    P.dv_dang[p] = make_float2(fmaf((float)P.Di[2], VZ, fmaf((float)P.Di[1], VY, (float)P.Di[0] * VX)),
                                               fmaf((float)P.Da[1], VY, (float)P.Da[0] * VX));
            }
        }
        int ix, iyf;
        const bool fast = key_coord_fp32(xe, mx, ix) && key_coord_fp32(ye, my, iyf);
        if (!fast) {
            // the reading in FP64: every product and sum rounded once
            double xp, yp;
            if (P.preprojected) {
                xp = (double)X;
                yp = (double)Y;
            } else {
                const double Xd = X, Yd = Y, Zd = Z;
                xp = __dadd_rn(__dadd_rn(__dmul_rn(P.R[0], Xd), __dmul_rn(P.R[1], Yd)), __dmul_rn(P.R[2], Zd));
                yp = __dadd_rn(__dadd_rn(__dmul_rn(P.R[3], Xd), __dmul_rn(P.R[4], Yd)), __dmul_rn(P.R[5], Zd));
            }
            const double u = __dmul_rn(__dsub_rn(xp, P.x_lo), P.inv_size);
            const double w = __dmul_rn(__dsub_rn(yp, P.y_lo), P.inv_size);
            ix = (u >= 0.0 && u < (double)P.nx) ? (int)u : -1;
            iyf = (w >= 0.0 && w < (double)P.ny) ? (int)w : -1;
        }
        const int nb = P.n_bands > 1 ? P.n_bands : 1;
        const int rows = P.rows > 0 ? P.rows : P.ny;
        int key;
        // the spaxel row on the whole field, then the row window
        const int iy = (iyf >= 0 && iyf < P.ny) ? iyf - P.row_lo : -1;
        if (ix >= 0 && ix < P.nx && iy >= 0 && iy < rows) {
            key = (iy * P.nx + ix) * nb;
            if (nb > 1) {
                int ia;
                float ta, dta;
                ssp_cell(log10f(P.age[p]), P.la_nodes, P.n_age, ia, ta, dta);
                key += age_band(ia, P.apb, nb);
            }
        } else {
            key = P.nx * rows * nb;
        }
        P.key[p] = key;
        if (P.pin_out) {
            PartRec r;
            r.mass = P.mass[p];
            r.age = P.age[p];
            r.Z = P.Zm[p];
            r.v = v;
            P.pin_out[p] = r;
        }
    }
}

// ----------------------------------------------------------------------------
// Exclusive scan of int32 (3 phases: block sums, scan of sums, block scans).
// ----------------------------------------------------------------------------
constexpr int kScanThreads = 1024;
constexpr int kScanItems = 4;
constexpr int kScanTile = kScanThreads * kScanItems;

__device__ __forceinline__ int block_exclusive_scan(int v, int* warp_tot, int* total) {
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    int x = v;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        int y = __shfl_up_sync(0xffffffffu, x, o);
        if (lane >= o) x += y;
    }
    if (lane == 31) warp_tot[wid] = x;
    __syncthreads();
    if (wid == 0) {
        int t = (lane < (int)(blockDim.x >> 5)) ? warp_tot[lane] : 0;
        int s = t;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            int y = __shfl_up_sync(0xffffffffu, s, o);
            if (lane >= o) s += y;
        }
        warp_tot[lane] = s - t;
        if (lane == 31) *total = s;
    }
    __syncthreads();
    int r = x - v + warp_tot[wid];
    __syncthreads();
    return r;
}

__global__ void k_scan_reduce(const int* __restrict__ in, long long n, int* __restrict__ sums) {
    __shared__ int wt[32];
    __shared__ int tot;
    long long base = (long long)blockIdx.x * kScanTile;
    int s = 0;
#pragma unroll
    for (int i = 0; i < kScanItems; ++i) {
        long long idx = base + (long long)i * kScanThreads + threadIdx.x;
        if (idx < n) s += in[idx];
    }
    block_exclusive_scan(s, wt, &tot);
    if (threadIdx.x == 0) sums[blockIdx.x] = tot;
}

__global__ void k_scan_sums(int* sums, int nb) {
    __shared__ int wt[32];
    __shared__ int tot;
    int carry = 0;
    for (int base = 0; base < nb; base += blockDim.x) {
        int i = base + threadIdx.x;
        int v = (i < nb) ? sums[i] : 0;
        int e = block_exclusive_scan(v, wt, &tot);
        if (i < nb) sums[i] = carry + e;
        carry += tot;
        __syncthreads();
    }
}

__global__ void k_scan_apply(const int* __restrict__ in, long long n, const int* __restrict__ sums,
                             int* __restrict__ out) {
    __shared__ int wt[32];
    __shared__ int tot;
    long long base = (long long)blockIdx.x * kScanTile + (long long)threadIdx.x * kScanItems;
    int v[kScanItems];
    int s = 0;
#pragma unroll
    for (int i = 0; i < kScanItems; ++i) {
        long long idx = base + i;
        v[i] = (idx < n) ? in[idx] : 0;
        s += v[i];
    }
    int e = block_exclusive_scan(s, wt, &tot) + sums[blockIdx.x];
#pragma unroll
    for (int i = 0; i < kScanItems; ++i) {
        long long idx = base + i;
        if (idx < n) out[idx] = e;
        e += v[i];
    }
}

size_t scan_scratch_ints(long long n) { return (size_t)((n + kScanTile - 1) / kScanTile) + 1; }

int launch_exclusive_scan(const int* in, int* out, long long n, int* scratch, cudaStream_t st) {
    if (n <= 0) return 0;
    int nb = (int)((n + kScanTile - 1) / kScanTile);
    k_scan_reduce<<<nb, kScanThreads, 0, st>>>(in, n, scratch);
    k_scan_sums<<<1, kScanThreads, 0, st>>>(scratch, nb);
    k_scan_apply<<<nb, kScanThreads, 0, st>>>(in, n, scratch, out);
    return 3;
}

// ----------------------------------------------------------------------------
// Stable LSD radix sort of (key, particle index), up to 9 bits per pass.
// Per pass: per-tile digit counts (digit-major), exclusive scan, then a stable
// scatter in which each warp ranks its keys in index order with match.any.
// ----------------------------------------------------------------------------
constexpr int kSortThreads = 256;
constexpr int kSortWarps = kSortThreads / 32;
constexpr int kSortRounds = 16;
constexpr int kSortTile = kSortThreads * kSortRounds;  // 4096 keys
constexpr int kMaxBuckets = 512;

__global__ void __launch_bounds__(kSortThreads) k_radix_hist(const int* __restrict__ keys, long long n, int shift,
                                                             int nbits, int n_tiles, int* __restrict__ counts) {
    __shared__ int hist[kMaxBuckets];
    const int nb = 1 << nbits, mask = nb - 1;
    for (int d = threadIdx.x; d < nb; d += blockDim.x) hist[d] = 0;
    __syncthreads();
    long long base = (long long)blockIdx.x * kSortTile;
    for (int i = threadIdx.x; i < kSortTile; i += blockDim.x) {
        long long idx = base + i;
        if (idx < n) atomicAdd(&hist[(keys[idx] >> shift) & mask], 1);
    }
    __syncthreads();
    for (int d = threadIdx.x; d < nb; d += blockDim.x) counts[(long long)d * n_tiles + blockIdx.x] = hist[d];
}

// Scatter of one tile: each warp ranks its keys in index order (match.any),
// the tile's keys are then placed in shared memory in (digit, index) order,
// and written out from there, so that consecutive threads write consecutive
// positions of a digit's run: the writes are coalesced runs instead of one
// scattered 4-byte write per key. The output positions are those of the
// per-key scatter (tile offset of the digit + keys of that digit before it in
// the tile): the sort is stable and its result does not depend on this
// staging.
__global__ void __launch_bounds__(kSortThreads) k_radix_scatter(const int* __restrict__ keys_in,
                                                                const int* __restrict__ vals_in, long long n,
                                                                int shift, int nbits, int n_tiles,
                                                                const int* __restrict__ offsets,
                                                                int* __restrict__ keys_out,
                                                                int* __restrict__ vals_out) {
    // wcnt is dead once the local positions are known: the staged keys reuse it
    __shared__ int wcnt[kSortWarps][kMaxBuckets];  // 16 KB = kSortTile ints
    __shared__ int s_val[kSortTile];
    __shared__ int s_dig0[kMaxBuckets];   // first local position of digit d
    __shared__ int s_goff[kMaxBuckets];   // the tile's global offset of digit d
    __shared__ int s_wsum[kSortWarps];
    static_assert(kSortWarps * kMaxBuckets >= kSortTile, "staging area");
    int* s_key = &wcnt[0][0];
    const int nb = 1 << nbits, mask = nb - 1;
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    for (int d = lane; d < nb; d += 32) wcnt[w][d] = 0;
    __syncwarp();
    const long long tile0 = (long long)blockIdx.x * kSortTile;
    const long long base = tile0 + (long long)w * (kSortTile / kSortWarps);
    const unsigned lt = (1u << lane) - 1u;
    int key[kSortRounds], rank[kSortRounds];
#pragma unroll
    for (int r = 0; r < kSortRounds; ++r) {
        long long idx = base + r * 32 + lane;
        bool valid = idx < n;
        int k = valid ? keys_in[idx] : 0;
        int d = valid ? ((k >> shift) & mask) : (nb + 1);
        unsigned peers = __match_any_sync(0xffffffffu, d);
        int before = valid ? wcnt[w][d] : 0;
        __syncwarp();
        int leader = 31 - __clz(peers);
        if (valid && lane == leader) wcnt[w][d] = before + __popc(peers);
        __syncwarp();
        key[r] = k;
        rank[r] = before + __popc(peers & lt);
    }
    __syncthreads();
    // per digit: the warps' exclusive prefix (in place) and the tile's count;
    // then the exclusive prefix of the counts over digits (two digits per thread)
    int cnt2[2] = {0, 0};
#pragma unroll
    for (int h = 0; h < 2; ++h) {
        const int d = 2 * threadIdx.x + h;
        if (d < nb) {
            int run = 0;
#pragma unroll
            for (int ww = 0; ww < kSortWarps; ++ww) {
                int t = wcnt[ww][d];
                wcnt[ww][d] = run;
                run += t;
            }
            cnt2[h] = run;
            s_goff[d] = offsets[(long long)d * n_tiles + blockIdx.x];
        }
    }
    int incl = cnt2[0] + cnt2[1];
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        const int y = __shfl_up_sync(0xffffffffu, incl, o);
        if (lane >= o) incl += y;
    }
    if (lane == 31) s_wsum[w] = incl;
    __syncthreads();
    int wpre = 0;
#pragma unroll
    for (int ww = 0; ww < kSortWarps; ++ww) wpre += (ww < w) ? s_wsum[ww] : 0;
    const int excl = wpre + incl - (cnt2[0] + cnt2[1]);
    if (2 * threadIdx.x < nb) s_dig0[2 * threadIdx.x] = excl;
    if (2 * threadIdx.x + 1 < nb) s_dig0[2 * threadIdx.x + 1] = excl + cnt2[0];
    __syncthreads();
    // local positions (wcnt still holds the warps' prefixes), then stage
    int lpos[kSortRounds];
#pragma unroll
    for (int r = 0; r < kSortRounds; ++r) {
        const long long idx = base + r * 32 + lane;
        const int d = (key[r] >> shift) & mask;
        lpos[r] = (idx < n) ? s_dig0[d] + wcnt[w][d] + rank[r] : -1;
    }
    __syncthreads();  // every warp is done with wcnt
#pragma unroll
    for (int r = 0; r < kSortRounds; ++r) {
        if (lpos[r] >= 0) {
            const long long idx = base + r * 32 + lane;
            s_key[lpos[r]] = key[r];
            s_val[lpos[r]] = vals_in ? vals_in[idx] : (int)idx;
        }
    }
    __syncthreads();
    const long long rem = n - tile0;
    const int n_valid = rem < kSortTile ? (int)rem : kSortTile;
    for (int i = threadIdx.x; i < n_valid; i += kSortThreads) {
        const int k = s_key[i];
        const int d = (k >> shift) & mask;
        const long long pos = (long long)s_goff[d] + (i - s_dig0[d]);
        keys_out[pos] = k;
        vals_out[pos] = s_val[i];
    }
}

// seg_off[s] = first sorted position with key >= s, for s in [0, n_keys]; the
// sorted keys are in [0, n_keys). One thread per segment boundary, each a
// binary search over the sorted keys, so that the work per thread is bounded
// however the particles are spread (a small galaxy in a large field leaves
// runs of hundreds of thousands of empty segments, which one thread per
// particle would write one after another).
__global__ void k_seg_bounds(const int* __restrict__ skeys, long long n, int n_keys, int* __restrict__ seg_off) {
    for (long long s = blockIdx.x * (long long)blockDim.x + threadIdx.x; s <= n_keys;
         s += (long long)gridDim.x * blockDim.x) {
        long long lo = 0, hi = n;
        while (lo < hi) {
            const long long mid = (lo + hi) >> 1;
            if (skeys[mid] < s) lo = mid + 1; else hi = mid;
        }
        seg_off[s] = (int)lo;
    }
}

size_t sort_scratch_ints(long long n) {
    long long n_tiles = (n + kSortTile - 1) / kSortTile;
    long long counts = n_tiles * kMaxBuckets;
    return (size_t)(2 * counts) + scan_scratch_ints(counts) + 16;
}

int launch_sort_by_key(const int* keys, long long n, int n_keys, int* keys_tmp, int* vals_tmp, int* keys_out,
                       int* perm_out, int* seg_off, int* scratch, cudaStream_t st) {
    int launches = 0;
    if (n > 0) {
        int bits = 1;
        while ((1ll << bits) < (long long)n_keys) ++bits;   // keys lie in [0, n_keys)
        int passes = (bits + 8) / 9;
        int per = (bits + passes - 1) / passes;
        int n_tiles = (int)((n + kSortTile - 1) / kSortTile);
        long long n_counts = (long long)n_tiles << per;
        int* counts = scratch;
        int* offs = scratch + n_counts;
        int* sscr = offs + n_counts;
        const int* kin = keys;
        const int* vin = nullptr;
        for (int ps = 0; ps < passes; ++ps) {
            int shift = ps * per;
            int nb = (ps == passes - 1) ? (bits - shift) : per;
            // ping-pong so that the last pass lands in keys_out / perm_out
            bool to_final = ((passes - 1 - ps) % 2) == 0;
            int* kout = to_final ? keys_out : keys_tmp;
            int* vout = to_final ? perm_out : vals_tmp;
            long long cnt = (long long)n_tiles << nb;
            k_radix_hist<<<n_tiles, kSortThreads, 0, st>>>(kin, n, shift, nb, n_tiles, counts);
            launches += 1 + launch_exclusive_scan(counts, offs, cnt, sscr, st);
            k_radix_scatter<<<n_tiles, kSortThreads, 0, st>>>(kin, vin, n, shift, nb, n_tiles, offs, kout, vout);
            ++launches;
            kin = kout;
            vin = vout;
        }
    }
    long long nt = ((long long)n_keys + 1 + 255) / 256;
    if (nt > 16ll * sm_count()) nt = 16ll * sm_count();
    k_seg_bounds<<<(int)nt, 256, 0, st>>>(keys_out, n, n_keys, seg_off);
    return launches + 1;
}

int launch_assign(const AssignParams& P, cudaStream_t st) {
    if (P.n <= 0) return 0;
    long long nb = (P.n + 255) / 256;
    if (nb > 16ll * sm_count()) nb = 16ll * sm_count();
    k_assign<<<(int)nb, 256, 0, st>>>(P);
    return 1;
}

}  // namespace rubix
