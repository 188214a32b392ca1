// sketch.cu -- sketching operators of Alg. 1 (sample step) on the device.
//
// Dense +-1 operator: generated inside the GEMM (gemm.cu); this file only
// writes it out explicitly (a test hook).  Sparse-sign operator (nnz nonzeros
// per column, the "fast sparse operator" the paper mentions for its tall
// predecessor, Sec. 2 remark): applied as a deterministic sparse x dense
// product, reading A once.
#include <climits>

#include "common.cuh"

namespace bq {

namespace {

constexpr int kMaxNnz = 64;

// Column j of the sparse-sign operator: nnz distinct rows with signs.  Draw t
// uses counter (j, 1+t, 0, 0); each output word w proposes row
// ((w >> 1) * d) >> 31 with sign -1 iff (w & 1); repeated rows are skipped.
// The draw is bounded at 2^22 counters (2^24 proposals).  For nnz <= d the
// chance that 2^24 uniform proposals miss one of nnz distinct rows is far
// below 2^-1000, so the bound is never reached; if it were, the column is
// completed with the smallest unused rows (sign +1), so that every row index
// stays in [0, d) whatever happens.  Returns nnz.
__device__ int sparse_column(uint64_t seed, i64 d, i64 j, int nnz, int* rows, double* sg) {
    int got = 0;
    for (uint32_t t = 0; got < nnz; ++t) {
        if (t > (1u << 22)) {
            for (int r = 0; got < nnz && r < d; ++r) {
                bool taken = false;
                for (int e = 0; e < got; ++e) taken |= (rows[e] == r);
                if (taken) continue;
                rows[got] = r;
                sg[got] = 1.0;
                ++got;
            }
            return got;
        }
        uint32_t o[4];
        philox4x32_10((uint32_t)j, 1u + t, 0u, 0u, (uint32_t)seed, (uint32_t)(seed >> 32), o);
#pragma unroll
        for (int q = 0; q < 4; ++q) {
            if (got >= nnz) break;
            const uint32_t w = o[q];
            const int row = (int)(((uint64_t)(w >> 1) * (uint64_t)d) >> 31);
            bool taken = false;
            for (int e = 0; e < got; ++e) taken |= (rows[e] == row);
            if (taken) continue;
            rows[got] = row;
            sg[got] = (w & 1u) ? -1.0 : 1.0;
            ++got;
        }
    }
    return got;
}

__global__ void dense_write_kernel(i64 d, i64 m, uint64_t seed, double* S, i64 lds) {
    const i64 total = d * m;
    for (i64 e = (i64)blockIdx.x * blockDim.x + threadIdx.x; e < total; e += (i64)gridDim.x * blockDim.x) {
        const i64 r = e % d, j = e / d;
        S[r + j * lds] = sketch_dense_entry(seed, r, j);
    }
}

__global__ void sparse_csc_kernel(i64 d, i64 m, uint64_t seed, int nnz, int* rows, double* sg) {
    const i64 j = (i64)blockIdx.x * blockDim.x + threadIdx.x;
    if (j >= m) return;
    int r[kMaxNnz];
    double s[kMaxNnz];
    sparse_column(seed, d, j, nnz, r, s);   // always nnz distinct rows in [0, d)
    for (int q = 0; q < nnz; ++q) {
        rows[j * nnz + q] = r[q];
        sg[j * nnz + q] = s[q];
    }
}

// One thread per column: zero it, then write its nnz signed entries.
__global__ void sparse_write_direct_kernel(i64 d, i64 m, uint64_t seed, int nnz, double* S, i64 lds) {
    const i64 j = (i64)blockIdx.x * blockDim.x + threadIdx.x;
    if (j >= m) return;
    for (i64 r = 0; r < d; ++r) S[r + j * lds] = 0.0;
    int r[kMaxNnz];
    double s[kMaxNnz];
    sparse_column(seed, d, j, nnz, r, s);
    for (int q = 0; q < nnz; ++q) S[r[q] + j * lds] = s[q];
}

__global__ void count_rows_kernel(i64 m, int nnz, const int* rows, int* cnt) {
    const i64 e = (i64)blockIdx.x * blockDim.x + threadIdx.x;
    if (e >= m * nnz) return;
    atomicAdd(&cnt[rows[e]], 1);
}

// exclusive scan of cnt[0..d) into ptr[0..d], single block
__global__ void __launch_bounds__(1024) scan_kernel(i64 d, const int* cnt, int* ptr) {
    __shared__ int part[1024];
    const int tid = threadIdx.x;
    const i64 chunk = (d + 1023) / 1024;
    const i64 lo = tid * chunk, hi = (lo + chunk < d) ? lo + chunk : d;
    int s = 0;
    for (i64 r = lo; r < hi; ++r) s += cnt[r];
    part[tid] = s;
    __syncthreads();
    if (tid == 0) {
        int acc = 0;
        for (int q = 0; q < 1024; ++q) { const int v = part[q]; part[q] = acc; acc += v; }
        ptr[d] = acc;
    }
    __syncthreads();
    int acc = part[tid];
    for (i64 r = lo; r < hi; ++r) { ptr[r] = acc; acc += cnt[r]; }
}

__global__ void fill_rows_kernel(i64 m, int nnz, const int* rows, const double* sg, const int* ptr, int* fillc,
                                 int* col, double* val) {
    const i64 e = (i64)blockIdx.x * blockDim.x + threadIdx.x;
    if (e >= m * nnz) return;
    const int r = rows[e];
    const int at = ptr[r] + atomicAdd(&fillc[r], 1);
    col[at] = (int)(e / nnz);
    val[at] = sg[e];
}

// Sort each CSR row by column, so that the row's sum runs in increasing i
// whatever order the atomic fill produced (the columns of a row are distinct,
// so the sorted order is unique).  In-place heapsort: O(k log k) for a row of
// k entries (k is about m*nnz/d, up to m*nnz when d is small).
__device__ void sift_down(int* col, double* val, int root, int n) {
    while (true) {
        int child = 2 * root + 1;
        if (child >= n) return;
        if (child + 1 < n && col[child + 1] > col[child]) ++child;
        if (col[root] >= col[child]) return;
        const int tc = col[root];
        col[root] = col[child];
        col[child] = tc;
        const double tv = val[root];
        val[root] = val[child];
        val[child] = tv;
        root = child;
    }
}

__global__ void sort_rows_kernel(i64 d, const int* ptr, int* col, double* val) {
    const i64 r = (i64)blockIdx.x * blockDim.x + threadIdx.x;
    if (r >= d) return;
    const int lo = ptr[r], n = ptr[r + 1] - lo;
    int* c = col + lo;
    double* v = val + lo;
    for (int i = n / 2 - 1; i >= 0; --i) sift_down(c, v, i, n);
    for (int end = n - 1; end > 0; --end) {
        const int tc = c[0];
        c[0] = c[end];
        c[end] = tc;
        const double tv = v[0];
        v[0] = v[end];
        v[end] = tv;
        sift_down(c, v, 0, end);
    }
}

constexpr int SJ = 8;          // columns of A per CTA (each CSR entry feeds SJ FMAs)
constexpr int SI = 1024;       // rows of A per staged chunk
constexpr i64 kRowTile = 2048; // sketch rows per CTA (larger d is split over blockIdx.y)

// Msk(r, j) = sum over the CSR entries (i, s) of row r, in increasing i, of s*A(i, j).
// One thread per sketch row r; CTA (x, y) takes columns [SJ x, SJ x + SJ) of
// A and sketch rows [y rt, y rt + rt); its columns of A are staged in SI-row
// chunks (read once per row tile: once in all when d <= kRowTile).
__global__ void __launch_bounds__(1024) sparse_apply_kernel(i64 d, i64 rt, i64 m, i64 n, const double* __restrict__ A,
                                                            i64 lda, const int* __restrict__ ptr,
                                                            const int* __restrict__ col, const double* __restrict__ val,
                                                            double* Msk, i64 ldsk) {
    extern __shared__ double sm[];
    double* As = sm;                                  // [SJ][SI]
    double* acc = sm + SJ * SI;                       // [rt][SJ]
    int* cur = reinterpret_cast<int*>(acc + rt * SJ); // [rt]
    const i64 j0 = (i64)blockIdx.x * SJ;
    const int nj = (int)((j0 + SJ <= n) ? SJ : n - j0);
    const i64 r0 = (i64)blockIdx.y * rt;
    const i64 nr = (r0 + rt <= d) ? rt : d - r0;      // rows of this tile
    ptr += r0;
    Msk += r0;
    for (i64 r = threadIdx.x; r < nr; r += blockDim.x) {
        cur[r] = ptr[r];
        for (int q = 0; q < SJ; ++q) acc[r * SJ + q] = 0.0;
    }
    for (i64 i0 = 0; i0 < m; i0 += SI) {
        const int ni = (int)((i0 + SI <= m) ? SI : m - i0);
        __syncthreads();
        for (int e = threadIdx.x; e < SJ * SI; e += blockDim.x) {
            const int q = e / SI, i = e % SI;
            As[e] = (q < nj && i < ni) ? A[(i0 + i) + (j0 + q) * lda] : 0.0;
        }
        __syncthreads();
        for (i64 r = threadIdx.x; r < nr; r += blockDim.x) {
            int e = cur[r];
            const int end = ptr[r + 1];
            double a[SJ];
#pragma unroll
            for (int q = 0; q < SJ; ++q) a[q] = acc[r * SJ + q];
            while (e < end && col[e] < i0 + ni) {
                const int i = (int)(col[e] - i0);
                const double sv = val[e];
#pragma unroll
                for (int q = 0; q < SJ; ++q) a[q] = fma(sv, As[q * SI + i], a[q]);
                ++e;
            }
            cur[r] = e;
#pragma unroll
            for (int q = 0; q < SJ; ++q) acc[r * SJ + q] = a[q];
        }
    }
    __syncthreads();
    for (i64 r = threadIdx.x; r < nr; r += blockDim.x)
        for (int q = 0; q < nj; ++q) Msk[r + (j0 + q) * ldsk] = acc[r * SJ + q];
}

// Sketch rows per CTA: d split into equal tiles of at most kRowTile rows.
i64 sparse_row_tile(i64 d) { return cdiv(d, cdiv(d, kRowTile)); }
size_t sparse_smem(i64 rt) { return (size_t)SJ * SI * 8 + (size_t)rt * SJ * 8 + (size_t)rt * 4 + 64; }

struct SparseWs {
    int* rows;
    double* sg;
    int* cnt;
    int* ptr;
    int* fillc;
    int* col;
    double* val;
};

size_t carve_sparse(Arena& ar, i64 d, i64 m, i64 nnz, SparseWs* w) {
    const size_t e = (size_t)m * (size_t)nnz;
    w->rows = ar.take<int>(e);
    w->sg = ar.take<double>(e);
    w->cnt = ar.take<int>((size_t)d + 1);
    w->ptr = ar.take<int>((size_t)d + 1);
    w->fillc = ar.take<int>((size_t)d + 1);
    w->col = ar.take<int>(e);
    w->val = ar.take<double>(e);
    return ar.off;
}

int build_csc(const Ctx& c, i64 d, i64 m, uint64_t seed, i64 nnz, SparseWs& w) {
    sparse_csc_kernel<<<(unsigned)cdiv(m, 128), 128, 0, c.stream>>>(d, m, seed, (int)nnz, w.rows, w.sg);
    BQ_LAUNCH_CHECK();
    return 0;
}

}  // namespace

size_t sketch_sparse_ws(i64 d, i64 m, i64 nnz) {
    Arena ar;
    ar.dry = true;
    SparseWs w{};
    return carve_sparse(ar, d, m, nnz, &w);
}

int sketch_write(const Ctx& c, i64 d, i64 m, uint64_t seed, int kind, i64 nnz, double* S, i64 lds) {
    if (d <= 0 || m <= 0) return 0;
    if (kind == BQRRP_SKETCH_DENSE) {
        const int blocks = (int)imin(cdiv(d * m, 256), 16LL * c.dev.sms);
        dense_write_kernel<<<blocks, 256, 0, c.stream>>>(d, m, seed, S, lds);
        BQ_LAUNCH_CHECK();
        return 0;
    }
    if (nnz < 1 || nnz > kMaxNnz || nnz > d) { set_error("sparse sketch: bad nnz"); return BQRRP_EUNSUPPORTED; }
    sparse_write_direct_kernel<<<(unsigned)cdiv(m, 128), 128, 0, c.stream>>>(d, m, seed, (int)nnz, S, lds);
    BQ_LAUNCH_CHECK();
    return 0;
}

int sketch_sparse_apply(const Ctx& c, i64 d, i64 m, i64 n, uint64_t seed, i64 nnz, const double* A, i64 lda,
                        double* Msk, i64 ldsk, void* ws, size_t ws_bytes) {
    if (d <= 0 || n <= 0) return 0;
    if (nnz < 1 || nnz > kMaxNnz || nnz > d) { set_error("sparse sketch: bad nnz"); return BQRRP_EUNSUPPORTED; }
    if (d > (i64)1 << 30 || m * nnz >= (i64)1 << 31) { set_error("sparse sketch: shape too large"); return BQRRP_EUNSUPPORTED; }
    const i64 rt = sparse_row_tile(d);
    const size_t smem = sparse_smem(rt);
    Arena ar;
    ar.base = (char*)ws;
    ar.cap = ws_bytes;
    SparseWs w{};
    carve_sparse(ar, d, m, nnz, &w);
    if (!ar.ok()) { set_error("sparse sketch: workspace too small"); return BQRRP_ENOMEM; }
    BQ_TRY(build_csc(c, d, m, seed, nnz, w));
    BQ_CUDA(cudaMemsetAsync(w.cnt, 0, sizeof(int) * (size_t)(d + 1), c.stream));
    BQ_CUDA(cudaMemsetAsync(w.fillc, 0, sizeof(int) * (size_t)(d + 1), c.stream));
    const i64 e = m * nnz;
    count_rows_kernel<<<(unsigned)cdiv(e, 256), 256, 0, c.stream>>>(m, (int)nnz, w.rows, w.cnt);
    BQ_LAUNCH_CHECK();
    scan_kernel<<<1, 1024, 0, c.stream>>>(d, w.cnt, w.ptr);
    BQ_LAUNCH_CHECK();
    fill_rows_kernel<<<(unsigned)cdiv(e, 256), 256, 0, c.stream>>>(m, (int)nnz, w.rows, w.sg, w.ptr, w.fillc, w.col,
                                                                  w.val);
    BQ_LAUNCH_CHECK();
    sort_rows_kernel<<<(unsigned)cdiv(d, 128), 128, 0, c.stream>>>(d, w.ptr, w.col, w.val);
    BQ_LAUNCH_CHECK();
    BQ_TRY(kernel_attrs((const void*)sparse_apply_kernel, (int)sparse_smem(kRowTile)));
    const int threads = (int)imin(1024, cdiv(rt, 32) * 32);
    if (cdiv(n, SJ) > (i64)INT32_MAX) { set_error("sparse sketch: n too large"); return BQRRP_EUNSUPPORTED; }
    sparse_apply_kernel<<<dim3((unsigned)cdiv(n, SJ), (unsigned)cdiv(d, rt)), threads, smem, c.stream>>>(
        d, rt, m, n, A, lda, w.ptr, w.col, w.val, Msk, ldsk);
    BQ_LAUNCH_CHECK();
    return 0;
}

}  // namespace bq
