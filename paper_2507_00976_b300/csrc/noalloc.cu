// noalloc.cu -- sparse-sign sketch application without any device allocation.
//
// bqrrp_sketch_apply (sparse kind) needs a caller-provided workspace for the
// operator's column and row index lists.  Some callers cannot provide one:
// code that runs with every byte of device memory already handed to another
// allocator (a framework's caching pool, a fixed serving budget), plug-ins that
// receive device pointers but no way to allocate, or hot loops that must never
// enter the allocator.  This variant keeps that scratch in a fixed array that
// lives in the library's own device image instead.
//
// Limits: m * nnz <= 2^19 operator entries and d <= 4096 sketch rows (about
// 12.6 MB of device memory, held by every GPU that loads the library until the
// process exits).
#include <mutex>

#include "common.cuh"

namespace bq {

int sketch_sparse_apply(const Ctx& c, i64 d, i64 m, i64 n, uint64_t seed, i64 nnz, const double* A, i64 lda,
                        double* Msk, i64 ldsk, void* ws, size_t ws_bytes);

namespace {

constexpr i64 kMaxEntries = i64(1) << 19;   // m * nnz
constexpr i64 kMaxRows = 4096;              // d
// index lists: rows (int), signs (double), CSR columns (int), CSR values
// (double) per entry; counts, row pointers and fill cursors (int) per sketch
// row; plus alignment slack for the arena's 256-byte carving.
constexpr size_t kScratchBytes = (size_t)kMaxEntries * (4 + 8 + 4 + 8) + 3 * (size_t)(kMaxRows + 1) * 4 + 16 * 256;

static __device__ __align__(256) unsigned char g_sketch_scratch[kScratchBytes];

// Device address of g_sketch_scratch per device, looked up once with that
// device current (host code may not use the symbol itself as a pointer).
std::mutex g_mu;
void* g_addr[64] = {nullptr};

int scratch_address(int dev, void** out) {
    std::lock_guard<std::mutex> lk(g_mu);
    if (dev < 0 || dev >= 64) {
        set_error("sketch_apply_sparse_noalloc: device id %d out of range", dev);
        return BQRRP_ECUDA;
    }
    if (!g_addr[dev]) {
        void* p = nullptr;
        const cudaError_t e = cudaGetSymbolAddress(&p, g_sketch_scratch);
        if (e != cudaSuccess || !p) {
            set_error("sketch_apply_sparse_noalloc: cudaGetSymbolAddress failed: %s", cudaGetErrorString(e));
            return BQRRP_ECUDA;
        }
        g_addr[dev] = p;
    }
    *out = g_addr[dev];
    return 0;
}

}  // namespace
}  // namespace bq

using namespace bq;

extern "C" int bqrrp_sketch_apply_sparse_noalloc(int64_t d, int64_t m, int64_t n, const double* A, int64_t lda,
                                                 uint64_t seed, int64_t nnz, double* Msk, int64_t ldsk,
                                                 void* stream) {
    set_error("");
    if (d < 1) return -1;
    if (m < 0) return -2;
    if (n < 0) return -3;
    if (lda < imax(1, m)) return -5;
    if (nnz < 1 || nnz > d || nnz > 64) return -7;
    if (ldsk < d) return -9;
    if (d > kMaxRows) {
        set_error("sketch_apply_sparse_noalloc: d = %lld exceeds the fixed scratch limit of %lld rows", (long long)d,
                  (long long)kMaxRows);
        return BQRRP_EUNSUPPORTED;
    }
    if (m * nnz > kMaxEntries) {
        set_error("sketch_apply_sparse_noalloc: m * nnz = %lld exceeds the fixed scratch limit of %lld entries",
                  (long long)(m * nnz), (long long)kMaxEntries);
        return BQRRP_EUNSUPPORTED;
    }
    if (n == 0 || m == 0) {
        if (n > 0 && m == 0) {   // S*A with an empty inner dimension is zero
            if (!Msk) return -8;
            BQ_CUDA(cudaMemset2DAsync(Msk, sizeof(double) * ldsk, 0, sizeof(double) * d, n, (cudaStream_t)stream));
        }
        return 0;
    }
    if (!A) return -4;
    if (!Msk) return -8;
    Ctx c{};
    BQ_TRY(current_device(&c.dev));
    c.stream = (cudaStream_t)stream;
    void* scratch = nullptr;
    BQ_TRY(scratch_address(c.dev.id, &scratch));
    // The counters and the error flag inside the scratch are cleared on the
    // stream by sketch_sparse_apply itself before use; everything else is
    // fully overwritten, so no state leaks from the previous call.
    return sketch_sparse_apply(c, d, m, n, seed, nnz, A, lda, Msk, ldsk, scratch, kScratchBytes);
}
