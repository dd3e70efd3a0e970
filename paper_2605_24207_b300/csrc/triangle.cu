// Cyclic self-join (relnn_triangle_*): the DHN triangle homomorphism of paper Sec. 5,
//   Out(n; sum(a_n * b_v * c_w)) :- E(n, v), E(v, w), E(w, n), H(n; a), H(v; b), H(w; c),
// element-wise products, bag semantics (every E row is a tuple, every H row of a key matches), the
// per-position transformations (Mu) applied to a, b, c beforehand, i.e. pushed below the join.
//
// Plan (content track, cached): H's build side gives every edge its two distinct-key indices
// (edges with a key missing from H are dropped); the edges are sorted twice, by (n, v) into
// out-adjacency lists and by (w, n) into in-adjacency lists (CSR over distinct keys). A triangle
// anchored at edge (n, v) closes at every w in out(v) ∩ in(n): a worst-case-optimal intersection of
// two sorted lists per edge instead of a binary join chain that would materialise the 2-paths. Each
// distinct w gives one record (n, v, w, mult) with mult = (copies of v->w) x (copies of w->n); the
// records come out grouped by n (edge order), so the output rows are a segmented sum.
//
// Because H rows of one key all match, the sum factorises per key: with A_k = sum of a over the
// rows of key k (likewise B, C), Out[n] = A_n * sum over records of mult * B_v * C_w. With unique H
// keys (A_k is one row) the records name H rows and a, b, c are read in place; otherwise the forward
// folds a, b, c to key rows first. It walks the records (warp per range, lane = d / 32 features, 4 records'
// rows in flight), multiplies a
// row's sum by A_n when it is emitted, and the SUM fix-up adds rows cut by range edges. The
// backward walks the records again: dB_v += mult g * C_w, dC_w += mult g * B_v (g = dOut_n * A_n)
// by f32 atomics, dA_n = dOut_n * (the row's sum); the key gradients are then broadcast to H rows.
#include <new>
#include <string>

#include "fwd.cuh"
#include "primitives.cuh"

using namespace relnn;

struct relnn_tri_s {
    int kt = RELNN_I32;
    int64_t n_h = 0, U = 0, n_edges = 0, n_valid = 0, n_rec = 0, n_out = 0;
    JoinTable H;
    DevBuf rec_n, rec_v, rec_w, rec_m, seg;  // records (int32) and their output rows
    DevBuf out_keys;                         // int64 [n_out]
    DevBuf fold;                             // f32 [3][U][d] key rows of a, b, c
    DevBuf gkey;                             // f32 [3][U][d] key-row gradients
    DevBuf carry, jobs, status;
    bool direct = false;  // H keys unique: the records name H rows and a, b, c are read in place
};

namespace relnn {
namespace {

int grid_of(int64_t n) { return (int)std::min<int64_t>(ceil_div(std::max<int64_t>(n, 1), 256), (int64_t)num_sms() * 8); }

// Distinct-key indices of both ends of every edge; flag = both present.
__global__ void edge_uid_kernel(JoinView j, const void* src, const void* dst, int64_t n, int kt, int32_t* us,
                                int32_t* ud, int32_t* flag) {
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
        const int32_t a = j.lookup(load_key(src, kt, i)), b = j.lookup(load_key(dst, kt, i));
        us[i] = a;
        ud[i] = b;
        flag[i] = (a >= 0 && b >= 0) ? 1 : 0;
    }
}

// Composite sort keys of the kept edges: (first << shift) | second, and the degree counts.
__global__ void edge_keys_kernel(const int32_t* us, const int32_t* ud, const int32_t* flag, const int32_t* pos,
                                 int64_t n, int shift, uint64_t* kout, uint64_t* kin, int32_t* vout, int32_t* vin,
                                 int32_t* deg_out, int32_t* deg_in) {
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
        if (!flag[i]) continue;
        const int64_t p = pos[i];
        kout[p] = ((uint64_t)(uint32_t)us[i] << shift) | (uint32_t)ud[i];
        kin[p] = ((uint64_t)(uint32_t)ud[i] << shift) | (uint32_t)us[i];
        vout[p] = 0;
        vin[p] = 0;
        atomicAdd(deg_out + us[i], 1);
        atomicAdd(deg_in + ud[i], 1);
    }
}

// Low half of the sorted composite keys: the adjacency list entries.
__global__ void low_half_kernel(const uint64_t* k, int64_t n, uint64_t mask, int32_t* out) {
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
        out[i] = (int32_t)(k[i] & mask);
}

// Walks out(v) and in(n) (sorted, with repeats) together; calls f(w, c1 * c2) per common w.
template <class Fn>
__device__ __forceinline__ void intersect(const int32_t* l1, int64_t n1, const int32_t* l2, int64_t n2, Fn&& f) {
    int64_t i = 0, j = 0;
    while (i < n1 && j < n2) {
        const int32_t x = l1[i], y = l2[j];
        if (x < y) {
            ++i;
        } else if (y < x) {
            ++j;
        } else {
            int64_t c1 = 0, c2 = 0;
            while (i < n1 && l1[i] == x) ++i, ++c1;
            while (j < n2 && l2[j] == x) ++j, ++c2;
            f(x, c1 * c2);
        }
    }
}

// One thread per sorted edge (n, v): count (emit == false) or write (emit == true) its records.
template <bool EMIT>
__global__ void tri_records_kernel(const uint64_t* kout, int64_t m, int shift, uint64_t mask, const int32_t* out_off,
                                   const int32_t* out_nbr, const int32_t* in_off, const int32_t* in_nbr,
                                   int32_t* cnt, const int64_t* rec_off, int32_t* rn, int32_t* rv, int32_t* rw,
                                   int32_t* rmult, int* status) {
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < m; i += (int64_t)gridDim.x * blockDim.x) {
        const int32_t n = (int32_t)(kout[i] >> shift), v = (int32_t)(kout[i] & mask);
        const int32_t* l1 = out_nbr + out_off[v];
        const int32_t* l2 = in_nbr + in_off[n];
        const int64_t n1 = out_off[v + 1] - out_off[v], n2 = in_off[n + 1] - in_off[n];
        if (!EMIT) {
            int64_t c = 0;
            intersect(l1, n1, l2, n2, [&](int32_t, int64_t) { ++c; });
            cnt[i] = (int32_t)c;
        } else {
            int64_t r = rec_off[i];
            intersect(l1, n1, l2, n2, [&](int32_t w, int64_t mult) {
                rn[r] = n;
                rv[r] = v;
                rw[r] = w;
                if (mult > 0x7fffffff) raise_status(status, RELNN_DEV_BOUNDS);
                rmult[r] = (int32_t)(mult > 0x7fffffff ? 0x7fffffff : mult);
                ++r;
            });
        }
    }
}

__global__ void widen_kernel(const int32_t* a, int64_t n, int64_t* b) {
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
        b[i] = a[i];
}

__global__ void present_kernel(const int32_t* rn, int64_t r, int32_t* present) {
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < r; i += (int64_t)gridDim.x * blockDim.x)
        present[rn[i]] = 1;
}

__global__ void rec_seg_kernel(const int32_t* rn, int64_t r, const int32_t* out_row, int32_t* seg) {
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < r; i += (int64_t)gridDim.x * blockDim.x)
        seg[i] = out_row[rn[i]];
}

__global__ void uid_to_row_kernel(const int32_t* rows_sorted, const int32_t* run_start, int64_t r, int32_t* rn,
                                  int32_t* rv, int32_t* rw) {
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < r; i += (int64_t)gridDim.x * blockDim.x) {
        rn[i] = rows_sorted[run_start[rn[i]]];
        rv[i] = rows_sorted[run_start[rv[i]]];
        rw[i] = rows_sorted[run_start[rw[i]]];
    }
}

__global__ void tri_keys_kernel(const int32_t* present, const int32_t* out_row, const int64_t* ukeys, int64_t U,
                                int64_t* keys) {
    for (int64_t u = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; u < U; u += (int64_t)gridDim.x * blockDim.x)
        if (present[u]) keys[out_row[u]] = ukeys[u];
}

// Key rows: X_u = sum of x over the H rows of key u (rows in ascending order), for x = a, b, c.
__global__ void fold_kernel(const void* a, const void* b, const void* c, int bf16, int d, const int32_t* run_start,
                            const int32_t* rows_sorted, int64_t U, float* out) {
    const int64_t total = 3 * U * d;
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < total; i += (int64_t)gridDim.x * blockDim.x) {
        const int which = (int)(i / (U * d));
        const int64_t rem = i - (int64_t)which * U * d;
        const int64_t u = rem / d;
        const int f = (int)(rem - u * d);
        const void* x = which == 0 ? a : (which == 1 ? b : c);
        float s = 0.f;
        for (int32_t p = run_start[u]; p < run_start[u + 1]; ++p) {
            const int64_t idx = (int64_t)rows_sorted[p] * d + f;
            s += bf16 ? bf16_to_f32(reinterpret_cast<const uint16_t*>(x)[idx]) : reinterpret_cast<const float*>(x)[idx];
        }
        out[i] = s;
    }
}

// H-row gradients from key-row gradients: dx[row] = G_u[uid(row)] for x = a, b, c.
__global__ void unfold_kernel(const float* G, const int32_t* rows_sorted, const int32_t* uid_of_pos, int64_t n_h,
                              int64_t U, int d, float* da, float* db, float* dc) {
    const int64_t total = 3 * n_h * d;
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < total; i += (int64_t)gridDim.x * blockDim.x) {
        const int which = (int)(i / (n_h * d));
        const int64_t rem = i - (int64_t)which * n_h * d;
        const int64_t p = rem / d;  // sorted position
        const int f = (int)(rem - p * d);
        float* dx = which == 0 ? da : (which == 1 ? db : dc);
        if (!dx) continue;
        dx[(int64_t)rows_sorted[p] * d + f] = G[((int64_t)which * U + uid_of_pos[p]) * d + f];
    }
}

struct TriArgs {
    const void *A, *B, *C;         // rows of a, b, c: folded key rows (f32) or, with unique H keys, the
                                   // caller's rows (the records then name H rows)
    const int32_t *rn, *rv, *rw, *rm, *seg;
    int64_t r;
    int d;
    float* out;                    // [n_out][d]
    float* carry;                  // [n_ranges][2][d]
    int64_t n_ranges;
    int range_tiles;
    const float* dout;
    float *dA, *dB, *dC;           // key-row gradients
};

// F consecutive floats (16-, 8- or 4-byte accesses by F).
template <int F>
__device__ __forceinline__ void ld4(const float* p, float (&x)[F]) {
    if (F >= 4) {
#pragma unroll
        for (int i = 0; i < F; i += 4) {
            const float4 u = __ldg(reinterpret_cast<const float4*>(p + i));
            x[i] = u.x; x[i + 1] = u.y; x[i + 2] = u.z; x[i + 3] = u.w;
        }
    } else if (F == 2) {
        const float2 u = __ldg(reinterpret_cast<const float2*>(p));
        x[0] = u.x; x[1] = u.y;
    } else {
        x[0] = __ldg(p);
    }
}

template <int F>
__device__ __forceinline__ void st4(float* p, const float (&x)[F]) {
    if (F >= 4) {
#pragma unroll
        for (int i = 0; i < F; i += 4) __stcg(reinterpret_cast<float4*>(p + i), make_float4(x[i], x[i + 1], x[i + 2], x[i + 3]));
    } else {
#pragma unroll
        for (int i = 0; i < F; ++i) __stcg(p + i, x[i]);
    }
}

template <int F>
__device__ __forceinline__ void add4(float* p, const float (&x)[F]) {
    if (F >= 4) {
#pragma unroll
        for (int i = 0; i < F; i += 4) atomicAdd(reinterpret_cast<float4*>(p + i), make_float4(x[i], x[i + 1], x[i + 2], x[i + 3]));
    } else if (F == 2) {
        atomicAdd(reinterpret_cast<float2*>(p), make_float2(x[0], x[1]));
    } else {
        atomicAdd(p, x[0]);
    }
}

// F consecutive elements of a row of a, b or c, as f32.
template <int F, bool BF16>
__device__ __forceinline__ void ldrow(const void* base, int64_t row, int d, int c0, float (&x)[F]) {
    if (!BF16) {
        ld4<F>(reinterpret_cast<const float*>(base) + row * d + c0, x);
        return;
    }
    const uint16_t* p = reinterpret_cast<const uint16_t*>(base) + row * d + c0;
    if (F == 8) {
        const uint4 u = __ldg(reinterpret_cast<const uint4*>(p));
        const uint32_t w[4] = {u.x, u.y, u.z, u.w};
#pragma unroll
        for (int i = 0; i < 4; ++i) {
            x[2 * i] = __uint_as_float(w[i] << 16);
            x[2 * i + 1] = __uint_as_float(w[i] & 0xffff0000u);
        }
    } else if (F == 4) {
        const uint2 u = __ldg(reinterpret_cast<const uint2*>(p));
        x[0] = __uint_as_float(u.x << 16);
        x[1] = __uint_as_float(u.x & 0xffff0000u);
        x[2] = __uint_as_float(u.y << 16);
        x[3] = __uint_as_float(u.y & 0xffff0000u);
    } else if (F == 2) {
        const uint32_t u = __ldg(reinterpret_cast<const uint32_t*>(p));
        x[0] = __uint_as_float(u << 16);
        x[1] = __uint_as_float(u & 0xffff0000u);
    } else {
        x[0] = __uint_as_float((uint32_t)__ldg(p) << 16);
    }
}

__global__ void narrow_keys_kernel(const int64_t* k, int64_t n, int32_t* out) {
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
        out[i] = (int32_t)k[i];
}

// Records whose B and C rows are loaded before any is used.
constexpr int kInFlight = 4;

// Forward walk (BWD = false) or backward walk (BWD = true) over the records of a range.
template <int F, bool BWD, bool BF16>
__global__ void __launch_bounds__(256) tri_walk_kernel(TriArgs a) {
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const int warps_total = gridDim.x * (blockDim.x >> 5);
    const int64_t span = (int64_t)a.range_tiles * 32;
    const int c0 = lane * F;
    for (int64_t rg = (int64_t)blockIdx.x * (blockDim.x >> 5) + warp; rg < a.n_ranges; rg += warps_total) {
        const int64_t r0 = rg * span, r1 = imin64(a.r, r0 + span);
        const int prev_seg = r0 > 0 ? a.seg[r0 - 1] : -1;
        const int next_seg = r1 < a.r ? a.seg[r1] : -1;
        int cur = -1, curn = 0;
        bool first = true;
        float acc[F], g[F], an[F];
#pragma unroll
        for (int i = 0; i < F; ++i) acc[i] = g[i] = an[i] = 0.f;
        auto flush = [&](bool last) {
            if (BWD) {
                // dA_n += dOut_n * (this piece's sum); pieces of a cut row add up
                float t[F];
#pragma unroll
                for (int i = 0; i < F; ++i) t[i] = acc[i] * g[i];  // g holds dOut_n here
                add4<F>(a.dA + (int64_t)curn * a.d + c0, t);
            } else {
                const bool split = (first && prev_seg == cur) || (last && next_seg == cur);
                float* dst = split ? a.carry + (rg * 2 + (first ? 0 : 1)) * a.d : a.out + (int64_t)cur * a.d;
                float t[F];
#pragma unroll
                for (int i = 0; i < F; ++i) t[i] = acc[i] * an[i];
                st4<F>(dst + c0, t);
            }
#pragma unroll
            for (int i = 0; i < F; ++i) acc[i] = 0.f;
            first = false;
        };
        for (int64_t b0 = r0; b0 < r1; b0 += 32) {
            const int nb = (int)imin64(32, r1 - b0);
            const bool tv = lane < nb;
            const int sv = tv ? a.seg[b0 + lane] : -1;
            const int nv = tv ? a.rn[b0 + lane] : 0;
            const int vv = tv ? a.rv[b0 + lane] : 0;
            const int wv = tv ? a.rw[b0 + lane] : 0;
            const float mv = tv ? (float)a.rm[b0 + lane] : 0.f;
            for (int j0 = 0; j0 < nb; j0 += kInFlight) {
                float bf[kInFlight][F], cf[kInFlight][F], mj[kInFlight];
                int sj[kInFlight], nj[kInFlight], vj[kInFlight], wj[kInFlight];
#pragma unroll
                for (int u = 0; u < kInFlight; ++u) {
                    const int j = j0 + u < nb ? j0 + u : nb - 1;
                    sj[u] = __shfl_sync(0xffffffffu, sv, j);
                    nj[u] = __shfl_sync(0xffffffffu, nv, j);
                    vj[u] = __shfl_sync(0xffffffffu, vv, j);
                    wj[u] = __shfl_sync(0xffffffffu, wv, j);
                    mj[u] = __shfl_sync(0xffffffffu, mv, j);
                    ldrow<F, BF16>(a.B, vj[u], a.d, c0, bf[u]);
                    ldrow<F, BF16>(a.C, wj[u], a.d, c0, cf[u]);
                }
#pragma unroll
                for (int u = 0; u < kInFlight; ++u) {
                    if (j0 + u >= nb) break;
                    if (sj[u] != cur) {
                        if (cur >= 0) flush(false);
                        cur = sj[u];
                        curn = nj[u];
                        if (BWD) {
                            float dn[F];
                            ld4<F>(a.dout + (int64_t)cur * a.d + c0, dn);
                            ldrow<F, BF16>(a.A, curn, a.d, c0, an);
#pragma unroll
                            for (int i = 0; i < F; ++i) g[i] = dn[i];
                        } else {
                            ldrow<F, BF16>(a.A, curn, a.d, c0, an);
                        }
                    }
                    if (BWD) {
                        float gb[F], gc[F];
#pragma unroll
                        for (int i = 0; i < F; ++i) {
                            const float ga = g[i] * an[i] * mj[u];  // mult * dOut_n * A_n
                            gb[i] = ga * cf[u][i];
                            gc[i] = ga * bf[u][i];
                            acc[i] = fmaf(mj[u] * bf[u][i], cf[u][i], acc[i]);
                        }
                        add4<F>(a.dB + (int64_t)vj[u] * a.d + c0, gb);
                        add4<F>(a.dC + (int64_t)wj[u] * a.d + c0, gc);
                    } else {
#pragma unroll
                        for (int i = 0; i < F; ++i) acc[i] = fmaf(mj[u] * bf[u][i], cf[u][i], acc[i]);
                    }
                }
            }
        }
        if (cur >= 0) flush(true);
    }
}

template <int F, bool BF16>
void size_ranges(TriArgs& a) {
    static int bps = 0;
    if (bps <= 0 && cudaOccupancyMaxActiveBlocksPerMultiprocessor(&bps, tri_walk_kernel<F, false, BF16>, 256, 0) != cudaSuccess) {
        (void)cudaGetLastError();
        bps = 1;
    }
    const int64_t n32 = ceil_div(a.r, 32);
    const int64_t resident = (int64_t)std::max(1, bps) * num_sms() * 8;
    a.range_tiles = (int)std::min<int64_t>(ceil_div(n32, resident), 1 << 20);
    a.n_ranges = ceil_div(n32, a.range_tiles);
}

template <int F, bool BF16>
relnn_status walk(relnn_tri_s* T, TriArgs& a, bool bwd, cudaStream_t st) {
    size_ranges<F, BF16>(a);
    const int grid = (int)std::min<int64_t>(ceil_div(a.n_ranges, 8), (int64_t)num_sms() * 8);
    if (!bwd) {
        RELNN_TRY(T->carry.alloc(sizeof(float) * 2 * (size_t)a.d * a.n_ranges));
        a.carry = T->carry.as<float>();
        { ProfToken pt = prof_begin(RELNN_PROF_FWD_FP32, st); tri_walk_kernel<F, false, BF16><<<grid, 256, 0, st>>>(a); note_launch(); prof_end(pt, st); }
        RELNN_CUDA(cudaGetLastError());
        RELNN_TRY(launch_fixup(a.seg, a.r, a.range_tiles * 32, a.n_ranges, a.carry, a.out, a.d, false, false, T->jobs, st));
    } else {
        { ProfToken pt = prof_begin(RELNN_PROF_BWD_FP32, st); tri_walk_kernel<F, true, BF16><<<grid, 256, 0, st>>>(a); note_launch(); prof_end(pt, st); }
        RELNN_CUDA(cudaGetLastError());
    }
    return RELNN_OK;
}

template <bool BF16>
relnn_status run_walk_t(relnn_tri_s* T, TriArgs& a, bool bwd, cudaStream_t st) {
    switch (a.d / 32) {  // lane = F = d / 32 consecutive features
        case 1: return walk<1, BF16>(T, a, bwd, st);
        case 2: return walk<2, BF16>(T, a, bwd, st);
        case 4: return walk<4, BF16>(T, a, bwd, st);
        default: return walk<8, BF16>(T, a, bwd, st);
    }
}

relnn_status run_walk(relnn_tri_s* T, TriArgs& a, bool bwd, bool bf16_rows, cudaStream_t st) {
    return bf16_rows ? run_walk_t<true>(T, a, bwd, st) : run_walk_t<false>(T, a, bwd, st);
}

relnn_status check_rows(relnn_tri_s* T, const void* a, const void* b, const void* c, relnn_float_t dtype, int d) {
    RELNN_CHECK_ARG(T, "triangle: null plan");
    RELNN_CHECK_ARG(d == 32 || d == 64 || d == 128 || d == 256, "triangle: d in {32, 64, 128, 256}");
    RELNN_CHECK_ARG(dtype == RELNN_F32 || dtype == RELNN_BF16, "triangle: bad dtype");
    RELNN_CHECK_ARG(T->n_h == 0 || (a && b && c), "triangle: null rows");
    RELNN_CHECK_ARG(((reinterpret_cast<uintptr_t>(a) | reinterpret_cast<uintptr_t>(b) | reinterpret_cast<uintptr_t>(c)) & 15u) == 0,
                    "triangle: rows must be 16-byte aligned");
    return RELNN_OK;
}

relnn_status fold_rows(relnn_tri_s* T, const void* a, const void* b, const void* c, relnn_float_t dtype, int d,
                       cudaStream_t st) {
    RELNN_TRY(T->fold.alloc(sizeof(float) * 3 * (size_t)std::max<int64_t>(T->U, 1) * d));
    if (T->U > 0)
        { fold_kernel<<<grid_of(3 * T->U * d), 256, 0, st>>>(a, b, c, dtype == RELNN_BF16, d, T->H.run_start.as<int32_t>(),
                                                            T->H.rows_sorted.as<int32_t>(), T->U, T->fold.as<float>()); note_launch(); }
    RELNN_CUDA(cudaGetLastError());
    return RELNN_OK;
}

// Rows the walk reads: the caller's (records name H rows when H's keys are unique) or the folded
// key rows.
TriArgs base_args(relnn_tri_s* T, int d, const void* a, const void* b, const void* c) {
    TriArgs t{};
    if (T->direct) {
        t.A = a;
        t.B = b;
        t.C = c;
    } else {
        const float* f = T->fold.as<float>();
        t.A = f;
        t.B = f + (size_t)T->U * d;
        t.C = f + 2 * (size_t)T->U * d;
    }
    t.rn = T->rec_n.as<int32_t>();
    t.rv = T->rec_v.as<int32_t>();
    t.rw = T->rec_w.as<int32_t>();
    t.rm = T->rec_m.as<int32_t>();
    t.seg = T->seg.as<int32_t>();
    t.r = T->n_rec;
    t.d = d;
    return t;
}

}  // namespace
}  // namespace relnn

extern "C" {

relnn_status relnn_triangle_plan(const relnn_tri_desc* desc, void* stream, relnn_tri_t* out) {
    RELNN_CHECK_ARG(desc && out, "triangle plan: null argument");
    *out = nullptr;
    RELNN_CHECK_ARG(desc->key_type == RELNN_I32 || desc->key_type == RELNN_I64, "triangle plan: bad key type");
    RELNN_CHECK_ARG(desc->n_h >= 0 && (desc->n_h == 0 || desc->d_h_ids), "triangle plan: bad H");
    RELNN_CHECK_ARG(desc->n_edges >= 0 && desc->n_edges < (1ll << 31) - 1 &&
                        (desc->n_edges == 0 || (desc->d_src && desc->d_dst)), "triangle plan: bad E");
    cudaStream_t st = (cudaStream_t)stream;
    relnn_tri_s* T = new (std::nothrow) relnn_tri_s();
    if (!T) return RELNN_ENOMEM;
    auto fail = [&](relnn_status s) {
        cudaStreamSynchronize(st);
        delete T;
        return s;
    };
#define TRI_TRY(expr)                        \
    do {                                     \
        relnn_status s_ = (expr);            \
        if (s_ != RELNN_OK) return fail(s_); \
    } while (0)
#define TRI_CUDA(expr)                                                   \
    do {                                                                 \
        cudaError_t e_ = (expr);                                         \
        if (e_ != cudaSuccess) {                                         \
            set_error(std::string("CUDA: ") + cudaGetErrorString(e_));   \
            return fail(RELNN_ECUDA);                                    \
        }                                                                \
    } while (0)
    T->kt = desc->key_type;
    T->n_h = desc->n_h;
    T->n_edges = desc->n_edges;
    TRI_TRY(T->status.alloc(sizeof(int) * kStatusInts));
    TRI_CUDA(cudaMemsetAsync(T->status.p, 0, sizeof(int) * kStatusInts, st));
    TRI_TRY(join_table_build(T->H, desc->d_h_ids, desc->n_h, desc->key_type, st));
    T->U = T->H.n_unique;
    const int64_t E = desc->n_edges, U = T->U;
    if (E == 0 || U == 0) {
        TRI_TRY(T->out_keys.alloc(sizeof(int64_t)));
        *out = T;
        return RELNN_OK;
    }
    // a: both ends' distinct keys; keep the edges whose keys are both in H
    DevBuf us, ud, flag, pos;
    TRI_TRY(us.alloc_tmp(sizeof(int32_t) * E, st));
    TRI_TRY(ud.alloc_tmp(sizeof(int32_t) * E, st));
    TRI_TRY(flag.alloc_tmp(sizeof(int32_t) * (E + 1), st));
    TRI_TRY(pos.alloc_tmp(sizeof(int32_t) * (E + 1), st));
    { edge_uid_kernel<<<grid_of(E), 256, 0, st>>>(T->H.view(), desc->d_src, desc->d_dst, E, T->kt, us.as<int32_t>(),
                                                  ud.as<int32_t>(), flag.as<int32_t>()); note_launch(); }
    TRI_TRY(exclusive_scan<int32_t>(flag.as<int32_t>(), pos.as<int32_t>(), E, pos.as<int32_t>() + E, st));
    int32_t M32 = 0;
    TRI_CUDA(cudaMemcpyAsync(&M32, pos.as<int32_t>() + E, sizeof(int32_t), cudaMemcpyDeviceToHost, st));
    TRI_CUDA(cudaStreamSynchronize(st));
    const int64_t M = M32;
    T->n_valid = M;
    // b: CSR out (sorted by (n, v)) and CSR in (sorted by (w, n)) over distinct keys
    const int shift = std::max(1, bit_length((uint64_t)U));
    const uint64_t mask = (1ull << shift) - 1;
    DevBuf kout, kin, kt1, vout, vin, vt1, dego, degi, offo, offi, nbro, nbri;
    const int64_t Mx = std::max<int64_t>(M, 1);
    TRI_TRY(kout.alloc_tmp(sizeof(uint64_t) * Mx, st));
    TRI_TRY(kin.alloc_tmp(sizeof(uint64_t) * Mx, st));
    TRI_TRY(kt1.alloc_tmp(sizeof(uint64_t) * Mx, st));
    TRI_TRY(vout.alloc_tmp(sizeof(int32_t) * Mx, st));
    TRI_TRY(vin.alloc_tmp(sizeof(int32_t) * Mx, st));
    TRI_TRY(vt1.alloc_tmp(sizeof(int32_t) * Mx, st));
    TRI_TRY(dego.alloc_tmp(sizeof(int32_t) * (U + 1), st));
    TRI_TRY(degi.alloc_tmp(sizeof(int32_t) * (U + 1), st));
    TRI_TRY(offo.alloc_tmp(sizeof(int32_t) * (U + 1), st));
    TRI_TRY(offi.alloc_tmp(sizeof(int32_t) * (U + 1), st));
    TRI_TRY(nbro.alloc_tmp(sizeof(int32_t) * Mx, st));
    TRI_TRY(nbri.alloc_tmp(sizeof(int32_t) * Mx, st));
    TRI_CUDA(cudaMemsetAsync(dego.p, 0, sizeof(int32_t) * (U + 1), st));
    TRI_CUDA(cudaMemsetAsync(degi.p, 0, sizeof(int32_t) * (U + 1), st));
    { edge_keys_kernel<<<grid_of(E), 256, 0, st>>>(us.as<int32_t>(), ud.as<int32_t>(), flag.as<int32_t>(), pos.as<int32_t>(),
                                                   E, shift, kout.as<uint64_t>(), kin.as<uint64_t>(), vout.as<int32_t>(),
                                                   vin.as<int32_t>(), dego.as<int32_t>(), degi.as<int32_t>()); note_launch(); }
    TRI_TRY((radix_sort_pairs<uint64_t, int32_t>(kout.as<uint64_t>(), vout.as<int32_t>(), kt1.as<uint64_t>(),
                                                 vt1.as<int32_t>(), M, 2 * shift, st)));
    TRI_TRY((radix_sort_pairs<uint64_t, int32_t>(kin.as<uint64_t>(), vin.as<int32_t>(), kt1.as<uint64_t>(),
                                                 vt1.as<int32_t>(), M, 2 * shift, st)));
    TRI_TRY(exclusive_scan<int32_t>(dego.as<int32_t>(), offo.as<int32_t>(), U + 1, nullptr, st));
    TRI_TRY(exclusive_scan<int32_t>(degi.as<int32_t>(), offi.as<int32_t>(), U + 1, nullptr, st));
    if (M > 0) {
        { low_half_kernel<<<grid_of(M), 256, 0, st>>>(kout.as<uint64_t>(), M, mask, nbro.as<int32_t>()); note_launch(); }
        { low_half_kernel<<<grid_of(M), 256, 0, st>>>(kin.as<uint64_t>(), M, mask, nbri.as<int32_t>()); note_launch(); }
    }
    // c: records per sorted out-edge (count, scan, emit)
    DevBuf cnt, roff;
    TRI_TRY(cnt.alloc_tmp(sizeof(int32_t) * (Mx + 1), st));
    TRI_TRY(roff.alloc_tmp(sizeof(int64_t) * (Mx + 1), st));
    TRI_CUDA(cudaMemsetAsync(cnt.p, 0, sizeof(int32_t) * (Mx + 1), st));
    if (M > 0)
        { tri_records_kernel<false><<<grid_of(M), 256, 0, st>>>(kout.as<uint64_t>(), M, shift, mask, offo.as<int32_t>(),
                                                                nbro.as<int32_t>(), offi.as<int32_t>(), nbri.as<int32_t>(),
                                                                cnt.as<int32_t>(), nullptr, nullptr, nullptr, nullptr,
                                                                nullptr, T->status.as<int>()); note_launch(); }
    DevBuf cnt64;
    TRI_TRY(cnt64.alloc_tmp(sizeof(int64_t) * (Mx + 1), st));
    { widen_kernel<<<grid_of(M + 1), 256, 0, st>>>(cnt.as<int32_t>(), M + 1, cnt64.as<int64_t>()); note_launch(); }
    TRI_TRY(exclusive_scan<int64_t>(cnt64.as<int64_t>(), roff.as<int64_t>(), M, roff.as<int64_t>() + M, st));
    int64_t R = 0;
    TRI_CUDA(cudaMemcpyAsync(&R, roff.as<int64_t>() + M, sizeof(int64_t), cudaMemcpyDeviceToHost, st));
    TRI_CUDA(cudaStreamSynchronize(st));
    if (R >= (1ll << 31) - 1) {
        set_error("triangle plan: more than 2^31 records");
        return fail(RELNN_ENOTSUP);
    }
    T->n_rec = R;
    const int64_t Rx = std::max<int64_t>(R, 1);
    TRI_TRY(T->rec_n.alloc(sizeof(int32_t) * Rx));
    TRI_TRY(T->rec_v.alloc(sizeof(int32_t) * Rx));
    TRI_TRY(T->rec_w.alloc(sizeof(int32_t) * Rx));
    TRI_TRY(T->rec_m.alloc(sizeof(int32_t) * Rx));
    TRI_TRY(T->seg.alloc(sizeof(int32_t) * Rx));
    if (R > 0)
        { tri_records_kernel<true><<<grid_of(M), 256, 0, st>>>(kout.as<uint64_t>(), M, shift, mask, offo.as<int32_t>(),
                                                               nbro.as<int32_t>(), offi.as<int32_t>(), nbri.as<int32_t>(),
                                                               nullptr, roff.as<int64_t>(), T->rec_n.as<int32_t>(),
                                                               T->rec_v.as<int32_t>(), T->rec_w.as<int32_t>(),
                                                               T->rec_m.as<int32_t>(), T->status.as<int>()); note_launch(); }
    // d: output rows = keys n with at least one record, ascending
    DevBuf present, orow;
    TRI_TRY(present.alloc_tmp(sizeof(int32_t) * (U + 1), st));
    TRI_TRY(orow.alloc_tmp(sizeof(int32_t) * (U + 1), st));
    TRI_CUDA(cudaMemsetAsync(present.p, 0, sizeof(int32_t) * (U + 1), st));
    if (R > 0) { present_kernel<<<grid_of(R), 256, 0, st>>>(T->rec_n.as<int32_t>(), R, present.as<int32_t>()); note_launch(); }
    TRI_TRY(exclusive_scan<int32_t>(present.as<int32_t>(), orow.as<int32_t>(), U, orow.as<int32_t>() + U, st));
    int32_t nout = 0;
    TRI_CUDA(cudaMemcpyAsync(&nout, orow.as<int32_t>() + U, sizeof(int32_t), cudaMemcpyDeviceToHost, st));
    TRI_TRY(T->out_keys.alloc(sizeof(int64_t) * (U + 1)));
    { tri_keys_kernel<<<grid_of(U), 256, 0, st>>>(present.as<int32_t>(), orow.as<int32_t>(), T->H.ukeys.as<int64_t>(), U,
                                                  T->out_keys.as<int64_t>()); note_launch(); }
    if (R > 0) { rec_seg_kernel<<<grid_of(R), 256, 0, st>>>(T->rec_n.as<int32_t>(), R, orow.as<int32_t>(), T->seg.as<int32_t>()); note_launch(); }
    // unique H keys: a key's rows are one row, so the records can name H rows and the forward reads
    // a, b, c in place (no folding)
    T->direct = (U == T->n_h);
    if (T->direct && R > 0)
        { uid_to_row_kernel<<<grid_of(R), 256, 0, st>>>(T->H.rows_sorted.as<int32_t>(), T->H.run_start.as<int32_t>(), R,
                                                       T->rec_n.as<int32_t>(), T->rec_v.as<int32_t>(),
                                                       T->rec_w.as<int32_t>()); note_launch(); }
    int dev_status = 0;
    TRI_CUDA(cudaMemcpyAsync(&dev_status, T->status.p, sizeof(int), cudaMemcpyDeviceToHost, st));
    TRI_CUDA(cudaStreamSynchronize(st));
    T->n_out = nout;
    if (dev_status) {
        set_device_error(dev_status);
        set_error("triangle plan: a record's multiplicity exceeds 2^31");
        return fail(RELNN_EDEVICE);
    }
#undef TRI_TRY
#undef TRI_CUDA
    *out = T;
    return RELNN_OK;
}

relnn_status relnn_triangle_info(relnn_tri_t t, int64_t* n_out, int64_t* n_records, int64_t* n_edges_kept) {
    RELNN_CHECK_ARG(t, "triangle info: null plan");
    if (n_out) *n_out = t->n_out;
    if (n_records) *n_records = t->n_rec;
    if (n_edges_kept) *n_edges_kept = t->n_valid;
    return RELNN_OK;
}

relnn_status relnn_triangle_out_keys(relnn_tri_t t, void* d_out_keys, void* stream) {
    RELNN_CHECK_ARG(t && (t->n_out == 0 || d_out_keys), "triangle out keys: null argument");
    if (t->n_out == 0) return RELNN_OK;
    cudaStream_t st = (cudaStream_t)stream;
    if (t->kt == RELNN_I64) {
        RELNN_CUDA(cudaMemcpyAsync(d_out_keys, t->out_keys.p, sizeof(int64_t) * t->n_out, cudaMemcpyDeviceToDevice, st));
        return RELNN_OK;
    }
    { narrow_keys_kernel<<<grid_of(t->n_out), 256, 0, st>>>(t->out_keys.as<int64_t>(), t->n_out,
                                                          reinterpret_cast<int32_t*>(d_out_keys)); note_launch(); }
    RELNN_CUDA(cudaGetLastError());
    return RELNN_OK;
}

relnn_status relnn_triangle_forward(relnn_tri_t T, const void* d_a, const void* d_b, const void* d_c, relnn_float_t dtype,
                                    int32_t d, float* d_out, void* stream) {
    RELNN_TRY(check_rows(T, d_a, d_b, d_c, dtype, d));
    if (T->n_out == 0) return RELNN_OK;
    RELNN_CHECK_ARG(d_out && (reinterpret_cast<uintptr_t>(d_out) & 15u) == 0, "triangle: null or unaligned output");
    cudaStream_t st = (cudaStream_t)stream;
    if (!T->direct) RELNN_TRY(fold_rows(T, d_a, d_b, d_c, dtype, d, st));
    TriArgs a = base_args(T, d, d_a, d_b, d_c);
    a.out = d_out;
    return run_walk(T, a, false, T->direct && dtype == RELNN_BF16, st);
}

relnn_status relnn_triangle_backward(relnn_tri_t T, const void* d_a, const void* d_b, const void* d_c, relnn_float_t dtype,
                                     int32_t d, const float* d_dout, float* d_da, float* d_db, float* d_dc, void* stream) {
    RELNN_TRY(check_rows(T, d_a, d_b, d_c, dtype, d));
    cudaStream_t st = (cudaStream_t)stream;
    const size_t rows = sizeof(float) * (size_t)T->n_h * d;
    if (T->n_out == 0 || T->U == 0) {
        for (float* x : {d_da, d_db, d_dc})
            if (x) RELNN_CUDA(cudaMemsetAsync(x, 0, rows, st));
        return RELNN_OK;
    }
    RELNN_CHECK_ARG(d_dout && (reinterpret_cast<uintptr_t>(d_dout) & 15u) == 0, "triangle: null or unaligned dOut");
    if (T->direct) {
        // the walk adds straight into the H-row gradients (scratch rows for the skipped ones)
        RELNN_CHECK_ARG(((reinterpret_cast<uintptr_t>(d_da) | reinterpret_cast<uintptr_t>(d_db) |
                          reinterpret_cast<uintptr_t>(d_dc)) & 15u) == 0, "triangle: gradients must be 16-byte aligned");
        const int missing = (d_da ? 0 : 1) + (d_db ? 0 : 1) + (d_dc ? 0 : 1);
        if (missing) RELNN_TRY(T->gkey.alloc(rows * missing));
        float* spare = T->gkey.as<float>();
        float* g[3] = {d_da, d_db, d_dc};
        for (float*& x : g)
            if (!x) {
                x = spare;
                spare += (size_t)T->n_h * d;
            }
        for (float* x : g) RELNN_CUDA(cudaMemsetAsync(x, 0, rows, st));
        TriArgs a = base_args(T, d, d_a, d_b, d_c);
        a.dout = d_dout;
        a.dA = g[0];
        a.dB = g[1];
        a.dC = g[2];
        return run_walk(T, a, true, dtype == RELNN_BF16, st);
    }
    RELNN_TRY(fold_rows(T, d_a, d_b, d_c, dtype, d, st));
    const size_t keyrows = sizeof(float) * 3 * (size_t)T->U * d;
    RELNN_TRY(T->gkey.alloc(keyrows));
    RELNN_CUDA(cudaMemsetAsync(T->gkey.p, 0, keyrows, st));
    TriArgs a = base_args(T, d, d_a, d_b, d_c);
    a.dout = d_dout;
    a.dA = T->gkey.as<float>();
    a.dB = a.dA + (size_t)T->U * d;
    a.dC = a.dA + 2 * (size_t)T->U * d;
    RELNN_TRY(run_walk(T, a, true, false, st));
    { unfold_kernel<<<grid_of(3 * T->n_h * d), 256, 0, st>>>(T->gkey.as<float>(), T->H.rows_sorted.as<int32_t>(),
                                                            T->H.uid_of_pos.as<int32_t>(), T->n_h, T->U, d, d_da, d_db,
                                                            d_dc); note_launch(); }
    RELNN_CUDA(cudaGetLastError());
    return RELNN_OK;
}

relnn_status relnn_triangle_destroy(relnn_tri_t t) {
    if (!t) return RELNN_OK;
    cudaDeviceSynchronize();
    delete t;
    return RELNN_OK;
}

}  // extern "C"
