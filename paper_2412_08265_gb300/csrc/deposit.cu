// deposit.cu -- SSP lookup, Doppler shift, resampling and per-spaxel sum
// (Sec. 3: "Each star spectrum is calculated as a lookup from a simple stellar
// population (SSP) library ... Doppler shifted ... resampling ... the stellar
// spectra in each spaxel are summed up").
//
// K3 (k_setup) turns each in-field particle, in spaxel-sorted order, into a
// 32-byte record: its four mass-scaled bilinear corner weights, the template
// row of the (ia, iz) corner and the affine map from output bin j to the
// fractional SSP node position t(j). K4 (k_deposit) is persistent: each CTA
// owns a contiguous, cost-balanced range of (wavelength tile, work item)
// pairs; for each tile it stages the SSP slab (all templates x the tile's
// node range plus a Doppler halo) in shared memory with TMA, and its warps
// accumulate whole items (<= chunk particles of one spaxel) in registers in a
// fixed particle order. Spaxels with more than `chunk` particles are split
// into several items whose FP32 partial rows K5 adds in FP64 in item order, so
// the cube is bitwise reproducible and no global atomics are used.
#include "common.cuh"
#include "kernels.h"

namespace rubix {

// ----------------------------------------------------------------------------
// K3: per-particle setup (sorted order).
// ----------------------------------------------------------------------------
__device__ __forceinline__ void ssp_cell(float q, const float* __restrict__ nodes, int n, int& i, float& t) {
    // half-open cell [node_i, node_i+1) holding q; clamped outside the grid
    if (n < 2 || !(q > nodes[0])) { i = 0; t = 0.f; return; }
    if (q >= nodes[n - 1]) { i = n - 2; t = 1.f; return; }
    int lo = 0, hi = n - 1;  // nodes[lo] <= q < nodes[hi]
    while (hi - lo > 1) {
        int mid = (lo + hi) >> 1;
        if (nodes[mid] <= q) lo = mid; else hi = mid;
    }
    i = lo;
    t = (q - nodes[lo]) / (nodes[lo + 1] - nodes[lo]);
}

__global__ void k_setup(SetupParams P) {
    const long long n_in = P.seg_off[P.n_s];
    if (n_in > P.n_cap) return;
    const int n_ls = P.ssp.n_ls;
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n_in;
         i += (long long)gridDim.x * blockDim.x) {
        const int p = P.perm[i];
        const float m = P.mass[p], age = P.age[p], Z = P.Z[p];
        const double v = P.v[p];
        int ia, iz;
        float ta, tz;
        ssp_cell(log10f(age), P.ssp.la_nodes, P.ssp.n_age, ia, ta);
        ssp_cell(log10f(Z), P.ssp.lz_nodes, P.ssp.n_Z, iz, tz);
        const float ms = (float)P.flux_scale * m;
        DepRec r;
        r.w[0] = ms * ((1.f - ta) * (1.f - tz));
        r.w[1] = ms * (ta * (1.f - tz));
        r.w[2] = ms * ((1.f - ta) * tz);
        r.w[3] = ms * (ta * tz);
        const int c0 = ia * P.ssp.n_Z + iz;
        // t(j) = ((l0 + j dl) / dop - ls0) / dls = B + j A   (FP64)
        const double dop = (1.0 + P.z_cosmo) * (1.0 + v / kC_kms);
        const double alpha = 1.0 / (dop * P.ssp.dls);
        const double B = P.l0 * alpha - P.ssp.ls0 / P.ssp.dls;
        const double A = P.dl * alpha;
        const double t_last = B + A * (double)(P.n_lambda - 1);
        int bi = 0;
        float bf = 0.f, a_hi = 0.f, a_lo = 0.f;
        if (!(dop > 0.0) || !(B < (double)n_ls) || !(t_last >= -1.0) || !(B > -32768.0)) {
            r.w[0] = r.w[1] = r.w[2] = r.w[3] = 0.f;  // contributes nothing to any bin
        } else {
            const double fb = floor(B);
            bi = (int)fb;
            bf = (float)(B - fb);
            const double ah = __longlong_as_double(__double_as_longlong(A) & ~((1ll << 42) - 1));
            a_hi = (float)ah;
            a_lo = (float)(A - ah);
        }
        r.c0_bi = (c0 << 16) | (bi & 0xffff);
        r.bf = bf;
        r.a_hi = a_hi;
        r.a_lo = a_lo;
        P.rec[i] = r;
        PartRec pr;
        pr.mass = m; pr.age = age; pr.Z = Z; pr.v = (float)v;
        P.prec[i] = pr;
    }
}

int launch_setup(const SetupParams& P, long long n_total, cudaStream_t st) {
    if (n_total <= 0) return 0;
    long long nb = (n_total + 255) / 256;
    if (nb > 152 * 16) nb = 152 * 16;
    k_setup<<<(int)nb, 256, 0, st>>>(P);
    return 1;
}

// ----------------------------------------------------------------------------
// Work items: one per <= chunk particles of a spaxel; empty spaxels get one
// empty item (its row is written as zeros).
// ----------------------------------------------------------------------------
__global__ void k_item_counts(ItemParams P) {
    for (int s = blockIdx.x * blockDim.x + threadIdx.x; s <= P.n_s; s += gridDim.x * blockDim.x) {
        if (s == P.n_s) { P.n_items[s] = 0; P.n_parts[s] = 0; continue; }
        int cnt = P.seg_off[s + 1] - P.seg_off[s];
        int ni = cnt > 0 ? (cnt + P.chunk - 1) / P.chunk : 1;
        P.n_items[s] = ni;
        P.n_parts[s] = ni > 1 ? ni : 0;
    }
}

__global__ void k_item_fill(ItemParams P) {
    for (int s = blockIdx.x * blockDim.x + threadIdx.x; s < P.n_s; s += gridDim.x * blockDim.x) {
        const int base = P.item_off[s], ni = P.item_off[s + 1] - base;
        const bool split = P.part_off[s + 1] > P.part_off[s];
        const int b0 = P.seg_off[s], e0 = P.seg_off[s + 1];
        for (int i = 0; i < ni; ++i) {
            if ((long long)base + i >= P.item_cap) { atomicOr(P.err, kErrBadItem); return; }
            Item it;
            it.spaxel = s;
            it.begin = b0 + i * P.chunk;
            it.end = min(b0 + (i + 1) * P.chunk, e0);
            it.part_row = split ? P.part_off[s] + i : -1;
            P.items[base + i] = it;
        }
    }
}

int launch_items(const ItemParams& P, cudaStream_t st) {
    int nb = (P.n_s + 1 + 255) / 256;
    if (nb > 4096) nb = 4096;
    k_item_counts<<<nb, 256, 0, st>>>(P);
    int l = 1;
    l += launch_exclusive_scan(P.n_items, P.item_off, P.n_s + 1, P.scan_scratch, st);
    l += launch_exclusive_scan(P.n_parts, P.part_off, P.n_s + 1, P.scan_scratch, st);
    k_item_fill<<<nb, 256, 0, st>>>(P);
    return l + 1;
}

// ----------------------------------------------------------------------------
// K4: deposit.
// ----------------------------------------------------------------------------
constexpr int kDepHeader = 128;  // mbarrier + counters; the slab starts 128-B aligned

size_t deposit_smem_bytes(int n_rows_alloc, int slab_w, int elem_bytes) {
    return kDepHeader + (size_t)n_rows_alloc * slab_w * elem_bytes;
}

// First item index i in [0, n] with items[i].begin + c0 * i >= x (items[n] is
// the virtual end with begin = n_in).
__device__ __forceinline__ long long item_lower_bound(const Item* __restrict__ items, long long n, long long n_in,
                                                      long long c0, long long x) {
    long long lo = 0, hi = n;
    while (lo < hi) {
        long long mid = (lo + hi) >> 1;
        long long pre = (long long)items[mid].begin + c0 * mid;
        if (pre < x) lo = mid + 1; else hi = mid;
    }
    (void)n_in;
    return lo;
}

template <typename T>
__device__ __forceinline__ float tpl_global(const T* __restrict__ tpl, int pitch, int n_ls, int row, int k) {
    return (k >= 0 && k < n_ls) ? TplTraits<T>::ld(tpl + (long long)row * pitch + k) : 0.f;
}

template <typename T, int R>
__global__ void __launch_bounds__(512, 1) k_deposit(const DepositParams P, const __grid_constant__ CUtensorMap tmap) {
    extern __shared__ __align__(1024) unsigned char smem[];
    uint64_t* bar = reinterpret_cast<uint64_t*>(smem);
    int* s_next = reinterpret_cast<int*>(smem + 16);
    T* slab = reinterpret_cast<T*>(smem + kDepHeader);

    const int lane = threadIdx.x & 31;
    const long long n_in = P.seg_off[P.n_s];
    const long long n_items = P.item_off[P.n_s];
    const long long C0 = P.cost_c0;
    const long long Ct = n_in + C0 * n_items;
    if (Ct <= 0) return;
    const long long total = Ct * P.n_tiles;
    const long long lo = total * blockIdx.x / gridDim.x;
    const long long hi = total * (blockIdx.x + 1) / gridDim.x;
    if (lo >= hi) return;

    if (threadIdx.x == 0) {
        mbar_init(bar, 1);
        fence_mbar_init();
    }
    __syncthreads();

    const T* __restrict__ tpl = reinterpret_cast<const T*>(P.ssp.tpl);
    const int pitch = P.ssp.pitch, n_ls = P.ssp.n_ls;
    const int da = (P.ssp.n_age > 1) ? P.ssp.n_Z : 0;
    const int dz = (P.ssp.n_Z > 1) ? 1 : 0;
    const int slab_w = P.slab_w;
    uint32_t phase = 0;

    for (long long t = lo / Ct; t < P.n_tiles && t * Ct < hi; ++t) {
        const long long a = max(lo - t * Ct, 0ll), b = min(hi - t * Ct, Ct);
        if (a >= b) continue;
        const int i_a = (int)item_lower_bound(P.items, n_items, n_in, C0, a);
        const int i_b = (int)item_lower_bound(P.items, n_items, n_in, C0, b);
        if (i_a >= i_b) continue;
        const int klo = P.tile_klo[t];

        __syncthreads();  // all warps are done with the previous slab
        if (threadIdx.x == 0) {
            *s_next = i_a;
            if (slab_w > 0) {
                fence_proxy_async_smem();
                mbar_arrive_expect_tx(bar, (uint32_t)(P.n_boxes * P.box_rows * slab_w * (int)sizeof(T)));
                for (int bx = 0; bx < P.n_boxes; ++bx)
                    tma_load_2d(slab + (size_t)bx * P.box_rows * slab_w, &tmap, bar, klo, bx * P.box_rows);
            }
        }
        bool ok = true;
        if (slab_w > 0) {
            ok = mbar_wait_bounded(bar, phase, 4000000000ll);
            phase ^= 1u;
        }
        if (__syncthreads_or(!ok)) {
            if (threadIdx.x == 0) atomicOr(P.err, kErrTmaTimeout);
            return;
        }

        const int j0 = (int)t * P.tile_w;
        while (true) {
            int it = 0;
            if (lane == 0) it = atomicAdd(s_next, 1);
            it = __shfl_sync(0xffffffffu, it, 0);
            if (it >= i_b) break;
            const Item I = P.items[it];
            float acc[R];
#pragma unroll
            for (int r = 0; r < R; ++r) acc[r] = 0.f;

            for (int q = I.begin; q < I.end; ++q) {
                const float4 w4 = reinterpret_cast<const float4*>(P.rec)[2 * q];
                const float4 g4 = reinterpret_cast<const float4*>(P.rec)[2 * q + 1];
                const int c0_bi = __float_as_int(g4.x);
                const int c0 = rec_c0(c0_bi), bi = rec_bi(c0_bi);
                const float bf = g4.y, a_hi = g4.z, a_lo = g4.w;
                int kk[R];
                float ff[R];
                bool inr = true;
#pragma unroll
                for (int r = 0; r < R; ++r) {
                    const int j = j0 + lane + 32 * r;
                    const float jf = (float)j;
                    const float pp = jf * a_hi;           // exact
                    const float pi = floorf(pp);
                    const float s = (pp - pi) + fmaf(jf, a_lo, bf);
                    const float fl = floorf(s);
                    ff[r] = s - fl;
                    kk[r] = bi + (int)pi + (int)fl - klo;
                    if (j < P.n_lambda) inr = inr && (kk[r] >= 0) && (kk[r] + 1 < slab_w);
                }
                if (__all_sync(0xffffffffu, inr)) {
                    const T* s00 = slab + c0 * slab_w;
                    const T* s10 = s00 + da * slab_w;
                    const T* s01 = s00 + dz * slab_w;
                    const T* s11 = s10 + dz * slab_w;
#pragma unroll
                    for (int r = 0; r < R; ++r) {
                        const int k = kk[r];
                        if (j0 + lane + 32 * r < P.n_lambda) {
                            const float m0 = w4.x * TplTraits<T>::ld(s00 + k) + w4.y * TplTraits<T>::ld(s10 + k) +
                                             w4.z * TplTraits<T>::ld(s01 + k) + w4.w * TplTraits<T>::ld(s11 + k);
                            const float m1 = w4.x * TplTraits<T>::ld(s00 + k + 1) +
                                             w4.y * TplTraits<T>::ld(s10 + k + 1) +
                                             w4.z * TplTraits<T>::ld(s01 + k + 1) +
                                             w4.w * TplTraits<T>::ld(s11 + k + 1);
                            acc[r] += fmaf(ff[r], m1 - m0, m0);
                        }
                    }
                } else {
                    if (lane == 0 && P.slow_count) atomicAdd(P.slow_count, 1ull);
#pragma unroll
                    for (int r = 0; r < R; ++r) {
                        const int k = kk[r] + klo;
                        if (j0 + lane + 32 * r < P.n_lambda) {
                            float m0 = 0.f, m1 = 0.f;
                            const int rows[4] = {c0, c0 + da, c0 + dz, c0 + da + dz};
                            const float ws[4] = {w4.x, w4.y, w4.z, w4.w};
#pragma unroll
                            for (int c = 0; c < 4; ++c) {
                                m0 += ws[c] * tpl_global(tpl, pitch, n_ls, rows[c], k);
                                m1 += ws[c] * tpl_global(tpl, pitch, n_ls, rows[c], k + 1);
                            }
                            acc[r] += fmaf(ff[r], m1 - m0, m0);
                        }
                    }
                }
            }
            if (I.part_row >= P.part_cap || I.spaxel < 0 || I.spaxel >= P.n_s) {
                if (lane == 0) atomicOr(P.err, kErrBadItem);
                continue;
            }
            float* dst = (I.part_row < 0) ? P.cube + (long long)I.spaxel * P.n_lambda
                                          : P.partials + (long long)I.part_row * P.n_lambda;
#pragma unroll
            for (int r = 0; r < R; ++r) {
                const int j = j0 + lane + 32 * r;
                if (j < P.n_lambda) dst[j] = acc[r];
            }
        }
    }
}

template <typename T>
static int launch_deposit_t(const DepositParams& P, const CUtensorMap* tmap, int n_ctas, int threads, size_t smem,
                            cudaStream_t st) {
    const int R = P.tile_w / 32;
    void (*fn)(const DepositParams, const CUtensorMap) = nullptr;
    switch (R) {
        case 1: fn = k_deposit<T, 1>; break;
        case 2: fn = k_deposit<T, 2>; break;
        case 3: fn = k_deposit<T, 3>; break;
        case 4: fn = k_deposit<T, 4>; break;
        case 5: fn = k_deposit<T, 5>; break;
        case 6: fn = k_deposit<T, 6>; break;
        case 7: fn = k_deposit<T, 7>; break;
        case 8: fn = k_deposit<T, 8>; break;
        default: return -1;
    }
    if (cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem) != cudaSuccess) return -1;
    fn<<<n_ctas, threads, smem, st>>>(P, *tmap);
    return 1;
}

int launch_deposit(const DepositParams& P, const CUtensorMap* tmap, int n_ctas, int threads, size_t smem,
                   cudaStream_t st) {
    switch (P.ssp.dtype) {
        case 0: return launch_deposit_t<float>(P, tmap, n_ctas, threads, smem, st);
        case 1: return launch_deposit_t<__nv_bfloat16>(P, tmap, n_ctas, threads, smem, st);
        case 2: return launch_deposit_t<__half>(P, tmap, n_ctas, threads, smem, st);
    }
    return -1;
}

// ----------------------------------------------------------------------------
// K5: rows of split spaxels = FP64 sum of their partial rows in item order.
// ----------------------------------------------------------------------------
__global__ void k_combine(const int* __restrict__ part_off, int n_s, int n_lambda, const float* __restrict__ partials,
                          float* __restrict__ cube) {
    for (int s = blockIdx.x; s < n_s; s += gridDim.x) {
        const int p0 = part_off[s], p1 = part_off[s + 1];
        if (p1 <= p0) continue;
        for (int j = threadIdx.x; j < n_lambda; j += blockDim.x) {
            double acc = 0.0;
            for (int r = p0; r < p1; ++r) acc += (double)partials[(long long)r * n_lambda + j];
            cube[(long long)s * n_lambda + j] = (float)acc;
        }
    }
}

int launch_combine(const int* part_off, int n_s, int n_lambda, const float* partials, float* cube,
                   cudaStream_t st) {
    int nb = n_s < 152 * 8 ? n_s : 152 * 8;
    if (nb < 1) return 0;
    k_combine<<<nb, 256, 0, st>>>(part_off, n_s, n_lambda, partials, cube);
    return 1;
}

}  // namespace rubix
