// bsvd_api.cu -- the C-ABI of libbsvd (see include/bsvd.h).
//
// Host side only: argument checks, choice of block width and path, shared-
// memory planning, grouping of pointer-array batches by shape, and kernel
// launches.  Every arithmetic step of the SVD runs in the CUDA kernels.
#include <cuda_runtime.h>

#include <algorithm>
#include <cstdint>
#include <cstring>
#include <map>
#include <new>
#include <utility>
#include <vector>

#include "bsvd.h"
#include "gesvj_fused.cuh"
#include "internal.h"

struct bsvd_handle_s {
    int last_arg = 0;
    int last_cuda = 0;
    int device = -1;
    int max_smem = 0;      // opt-in shared memory per block (bytes)
    int sm_count = 0;
};

namespace {

using bsvd::FusedArgs;

constexpr double kU32 = 5.9604644775390625e-08;     // 2^-24
constexpr double kU64 = 1.1102230246251565e-16;     // 2^-53
constexpr int kDefaultMaxSweeps = 40;

bsvd_status fail_arg(bsvd_handle h, int pos) {
    if (h) h->last_arg = pos;
    return BSVD_ERR_INVALID;
}

bsvd_status fail_cuda(bsvd_handle h, cudaError_t e) {
    if (h) h->last_cuda = (int)e;
    return BSVD_ERR_CUDA;
}

bsvd_status refresh_device(bsvd_handle h) {
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return fail_cuda(h, e);
    if (dev != h->device) {
        e = cudaDeviceGetAttribute(&h->max_smem, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev);
        if (e != cudaSuccess) return fail_cuda(h, e);
        e = cudaDeviceGetAttribute(&h->sm_count, cudaDevAttrMultiProcessorCount, dev);
        if (e != cudaSuccess) return fail_cuda(h, e);
        h->device = dev;
    }
    return BSVD_OK;
}

struct Resolved {
    int nb, max_sweeps, inner_sweeps, path, flags;
    double tol;
};

// Options with defaults filled in.  Returns false for an invalid option.
bool resolve(const bsvd_opts* o, bool single, int N, Resolved& r) {
    bsvd_opts z;
    std::memset(&z, 0, sizeof z);
    if (!o) o = &z;
    if (o->nb < 0 || o->max_sweeps < 0 || o->inner_sweeps < 0 || o->tol < 0 || o->path < 0 ||
        o->path > BSVD_PATH_PLAIN)
        return false;
    r.nb = o->nb ? o->nb : (N >= 48 ? 16 : (N >= 12 ? 8 : 4));
    r.max_sweeps = o->max_sweeps ? o->max_sweeps : kDefaultMaxSweeps;
    r.max_sweeps = std::min(r.max_sweeps, bsvd::kMaxSweeps);
    r.inner_sweeps = o->inner_sweeps ? o->inner_sweeps : 1;
    r.tol = o->tol > 0 ? o->tol : 30.0 * (single ? kU32 : kU64);
    r.path = o->path;
    r.flags = o->flags;
    return true;
}

typedef size_t (*plan_fn)(int, int, int, bool, FusedArgs&, int&);
typedef cudaError_t (*launch_fn)(int, const FusedArgs&, int, size_t, cudaStream_t);

struct TypeOps {
    bool single;
    size_t elt;
    plan_fn plan;
    launch_fn launch;
};

TypeOps ops_for(char t) {
    switch (t) {
        case 's': return {true, 4, bsvd::fused_plan_s, bsvd::fused_launch_s};
        case 'd': return {false, 8, bsvd::fused_plan_d, bsvd::fused_launch_d};
        case 'c': return {true, 8, bsvd::fused_plan_c, bsvd::fused_launch_c};
        default:  return {false, 16, bsvd::fused_plan_z, bsvd::fused_launch_z};
    }
}

// One group of equal-shape matrices, planned for the fused kernel.
struct Plan {
    FusedArgs a;
    size_t smem = 0;
    int threads = 0;
    int nb = 0;
};

bsvd_status plan_group(bsvd_handle h, const TypeOps& ops, int m, int n, bool wantU, bool wantV,
                       const Resolved& r, Plan& p) {
    std::memset(&p.a, 0, sizeof p.a);
    FusedArgs& a = p.a;
    a.m = m;
    a.n = n;
    a.trans = m < n;
    a.M = std::max(m, n);
    a.N = std::min(m, n);
    a.wantU = wantU;
    a.wantV = wantV;
    a.tol = r.tol;
    a.max_sweeps = r.max_sweeps;
    a.inner_sweeps = r.inner_sweeps;
    a.flags = r.flags;
    const bool needVs = a.trans ? wantU : wantV;
    if (r.path == BSVD_PATH_PLAIN) return BSVD_ERR_NOT_IMPLEMENTED;
    p.nb = r.nb;
    p.smem = ops.plan(r.nb, a.M, a.N, needVs, a, p.threads);
    if (p.smem == 0) return BSVD_ERR_NOT_IMPLEMENTED;       // unsupported nb
    if (p.smem > (size_t)h->max_smem) return BSVD_ERR_NOT_IMPLEMENTED;   // does not fit on chip
    return BSVD_OK;
}

// Workspace of the pointer-array form: lda, ldu, ldv (3 x batch ints) plus
// the matrix ids grouped by shape (batch ints).
size_t batched_ws(int batch) { return ((size_t)4 * batch * sizeof(int) + 255) & ~size_t(255); }

bsvd_status strided_impl(char t, bsvd_handle h, bsvd_job jobu, bsvd_job jobv, int batch, int m,
                         int n, const void* dA, int lda, long long sA, void* dS, long long sS,
                         void* dU, int ldu, long long sU, void* dV, int ldv, long long sV,
                         int* d_info, int* d_sweeps, void* d_work, size_t work_bytes,
                         const bsvd_opts* opts, void* stream) {
    if (!h) return BSVD_ERR_INVALID;
    h->last_arg = 0;
    const int k = std::min(m, n);
    if (jobu != BSVD_JOB_NONE && jobu != BSVD_JOB_SOME) return fail_arg(h, 2);
    if (jobv != BSVD_JOB_NONE && jobv != BSVD_JOB_SOME) return fail_arg(h, 3);
    if (batch < 0) return fail_arg(h, 4);
    if (m < 0) return fail_arg(h, 5);
    if (n < 0) return fail_arg(h, 6);
    const bool wantU = jobu == BSVD_JOB_SOME, wantV = jobv == BSVD_JOB_SOME;
    if (batch > 0 && m > 0 && n > 0 && !dA) return fail_arg(h, 7);
    if (lda < std::max(1, m)) return fail_arg(h, 8);
    if (batch > 1 && sA < (long long)lda * n) return fail_arg(h, 9);
    if (batch > 0 && k > 0 && !dS) return fail_arg(h, 10);
    if (batch > 1 && sS < k) return fail_arg(h, 11);
    if (wantU && batch > 0 && k > 0 && !dU) return fail_arg(h, 12);
    if (wantU && ldu < std::max(1, m)) return fail_arg(h, 13);
    if (wantU && batch > 1 && sU < (long long)ldu * k) return fail_arg(h, 14);
    if (wantV && batch > 0 && k > 0 && !dV) return fail_arg(h, 15);
    if (wantV && ldv < std::max(1, n)) return fail_arg(h, 16);
    if (wantV && batch > 1 && sV < (long long)ldv * k) return fail_arg(h, 17);
    if (batch > 0 && !d_info) return fail_arg(h, 18);
    (void)d_work;
    (void)work_bytes;
    const TypeOps ops = ops_for(t);
    Resolved r;
    if (!resolve(opts, ops.single, k, r)) return fail_arg(h, 22);
    if (batch == 0) return BSVD_OK;
    bsvd_status st = refresh_device(h);
    if (st != BSVD_OK) return st;
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    if (k == 0) {   // empty matrices: nothing to compute, converged by definition
        cudaError_t e = cudaMemsetAsync(d_info, 0, sizeof(int) * (size_t)batch, s);
        if (e == cudaSuccess && d_sweeps) e = cudaMemsetAsync(d_sweeps, 0, sizeof(int) * (size_t)batch, s);
        return e == cudaSuccess ? BSVD_OK : fail_cuda(h, e);
    }
    Plan p;
    st = plan_group(h, ops, m, n, wantU, wantV, r, p);
    if (st != BSVD_OK) return st;
    FusedArgs& a = p.a;
    a.A = dA; a.sA = sA; a.lda = lda;
    a.S = dS; a.sS = sS;
    a.U = dU; a.sU = sU; a.ldu = ldu;
    a.V = dV; a.sV = sV; a.ldv = ldv;
    a.info = d_info;
    a.sweeps = d_sweeps;
    cudaError_t e = ops.launch(p.nb, a, batch, p.smem, s);
    return e == cudaSuccess ? BSVD_OK : fail_cuda(h, e);
}

bsvd_status batched_impl(char t, bsvd_handle h, bsvd_job jobu, bsvd_job jobv, int batch,
                         const int* m, const int* n, const void* const* dA, const int* lda,
                         void* const* dS, void* const* dU, const int* ldu, void* const* dV,
                         const int* ldv, int* d_info, int* d_sweeps, void* d_work,
                         size_t work_bytes, const bsvd_opts* opts, void* stream) {
    if (!h) return BSVD_ERR_INVALID;
    h->last_arg = 0;
    if (jobu != BSVD_JOB_NONE && jobu != BSVD_JOB_SOME) return fail_arg(h, 2);
    if (jobv != BSVD_JOB_NONE && jobv != BSVD_JOB_SOME) return fail_arg(h, 3);
    if (batch < 0) return fail_arg(h, 4);
    if (batch == 0) return BSVD_OK;
    const bool wantU = jobu == BSVD_JOB_SOME, wantV = jobv == BSVD_JOB_SOME;
    if (!m) return fail_arg(h, 5);
    if (!n) return fail_arg(h, 6);
    if (!dA) return fail_arg(h, 7);
    if (!lda) return fail_arg(h, 8);
    if (!dS) return fail_arg(h, 9);
    if (wantU && (!dU || !ldu)) return fail_arg(h, !dU ? 10 : 11);
    if (wantV && (!dV || !ldv)) return fail_arg(h, !dV ? 12 : 13);
    if (!d_info) return fail_arg(h, 14);
    for (int i = 0; i < batch; ++i) {
        if (m[i] < 0) return fail_arg(h, 5);
        if (n[i] < 0) return fail_arg(h, 6);
        if (lda[i] < std::max(1, m[i])) return fail_arg(h, 8);
        if (wantU && ldu[i] < std::max(1, m[i])) return fail_arg(h, 11);
        if (wantV && ldv[i] < std::max(1, n[i])) return fail_arg(h, 13);
    }
    const size_t need = batched_ws(batch);
    if (!d_work && work_bytes > 0) return fail_arg(h, 16);
    if (work_bytes < need || !d_work) return BSVD_ERR_WORKSPACE;
    if ((reinterpret_cast<uintptr_t>(d_work) & 15) != 0) return fail_arg(h, 16);
    const TypeOps ops = ops_for(t);
    bsvd_status st = refresh_device(h);
    if (st != BSVD_OK) return st;
    cudaStream_t s = static_cast<cudaStream_t>(stream);

    // group matrix ids by shape
    std::map<std::pair<int, int>, std::vector<int>> groups;
    for (int i = 0; i < batch; ++i) groups[{m[i], n[i]}].push_back(i);
    std::vector<int> host((size_t)4 * batch);
    std::memcpy(host.data(), lda, sizeof(int) * batch);
    for (int i = 0; i < batch; ++i) {
        host[batch + i] = wantU ? ldu[i] : 1;
        host[2 * batch + i] = wantV ? ldv[i] : 1;
    }
    size_t pos = 3 * (size_t)batch;
    std::vector<std::pair<size_t, const std::vector<int>*>> order;
    for (auto& kv : groups) {
        order.push_back({pos, &kv.second});
        std::copy(kv.second.begin(), kv.second.end(), host.begin() + pos);
        pos += kv.second.size();
    }
    // plan every group before touching the device, so a bad shape fails cleanly
    std::vector<Plan> plans(groups.size());
    size_t gi = 0;
    for (auto& kv : groups) {
        const int mm = kv.first.first, nn = kv.first.second;
        Resolved r;
        if (!resolve(opts, ops.single, std::min(mm, nn), r)) return fail_arg(h, 18);
        if (std::min(mm, nn) > 0) {
            st = plan_group(h, ops, mm, nn, wantU, wantV, r, plans[gi]);
            if (st != BSVD_OK) return st;
        }
        ++gi;
    }
    int* dws = static_cast<int*>(d_work);
    cudaError_t e = cudaMemcpyAsync(dws, host.data(), sizeof(int) * host.size(), cudaMemcpyHostToDevice, s);
    if (e != cudaSuccess) return fail_cuda(h, e);
    gi = 0;
    for (auto& kv : groups) {
        const int mm = kv.first.first, nn = kv.first.second;
        const int count = (int)kv.second.size();
        const size_t ipos = order[gi].first;
        Plan& p = plans[gi++];
        if (std::min(mm, nn) == 0) {
            // zero-size matrices: info = 0 (written by a tiny memset per id is
            // awkward; set through the fused kernel's tail instead is overkill)
            for (int id : kv.second) {
                e = cudaMemsetAsync(d_info + id, 0, sizeof(int), s);
                if (e == cudaSuccess && d_sweeps) e = cudaMemsetAsync(d_sweeps + id, 0, sizeof(int), s);
                if (e != cudaSuccess) return fail_cuda(h, e);
            }
            continue;
        }
        FusedArgs& a = p.a;
        a.Ap = dA; a.ldap = dws;
        a.Sp = dS;
        a.Up = dU; a.ldup = dws + batch;
        a.Vp = dV; a.ldvp = dws + 2 * batch;
        a.index = dws + ipos;
        a.info = d_info;
        a.sweeps = d_sweeps;
        e = ops.launch(p.nb, a, count, p.smem, s);
        if (e != cudaSuccess) return fail_cuda(h, e);
    }
    return BSVD_OK;
}

}  // namespace

extern "C" {

bsvd_status bsvd_create(bsvd_handle* handle) {
    if (!handle) return BSVD_ERR_INVALID;
    *handle = new (std::nothrow) bsvd_handle_s();
    return *handle ? BSVD_OK : BSVD_ERR_NOMEM;
}

bsvd_status bsvd_destroy(bsvd_handle handle) {
    delete handle;
    return BSVD_OK;
}

const char* bsvd_status_string(bsvd_status s) {
    switch (s) {
        case BSVD_OK: return "BSVD_OK";
        case BSVD_ERR_INVALID: return "BSVD_ERR_INVALID: invalid argument";
        case BSVD_ERR_WORKSPACE: return "BSVD_ERR_WORKSPACE: workspace too small";
        case BSVD_ERR_CUDA: return "BSVD_ERR_CUDA: a CUDA call failed";
        case BSVD_ERR_TIMEOUT: return "BSVD_ERR_TIMEOUT: a bounded device wait expired";
        case BSVD_ERR_NOT_IMPLEMENTED: return "BSVD_ERR_NOT_IMPLEMENTED: shape/type/option not supported";
        case BSVD_ERR_NOMEM: return "BSVD_ERR_NOMEM: host allocation failed";
    }
    return "unknown bsvd_status";
}

int bsvd_last_arg(bsvd_handle h) { return h ? h->last_arg : 0; }
int bsvd_last_cuda(bsvd_handle h) { return h ? h->last_cuda : 0; }
int bsvd_version(void) { return BSVD_VERSION; }

bsvd_status bsvd_gesvj_workspace(bsvd_handle handle, char dtype, int batch, const int* m_arr,
                                 const int* n_arr, int uniform, bsvd_job jobu, bsvd_job jobv,
                                 const bsvd_opts* opts, size_t* bytes) {
    if (!handle) return BSVD_ERR_INVALID;
    handle->last_arg = 0;
    if (dtype != 's' && dtype != 'd' && dtype != 'c' && dtype != 'z') return fail_arg(handle, 2);
    if (batch < 0) return fail_arg(handle, 3);
    if (batch > 0 && (!m_arr || !n_arr)) return fail_arg(handle, !m_arr ? 4 : 5);
    if (!bytes) return fail_arg(handle, 10);
    (void)jobu;
    (void)jobv;
    (void)opts;
    *bytes = (uniform || batch == 0) ? 0 : batched_ws(batch);
    return BSVD_OK;
}

#define BSVD_STRIDED_IMPL(TAG, T, R)                                                          \
    bsvd_status bsvd_##TAG##gesvj_strided(BSVD_STRIDED_ARGS(T, R)) {                           \
        return strided_impl(#TAG[0], handle, jobu, jobv, batch, m, n, dA, lda, strideA, dS,    \
                            strideS, dU, ldu, strideU, dV, ldv, strideV, d_info, d_sweeps,     \
                            d_work, work_bytes, opts, stream);                                 \
    }
BSVD_STRIDED_IMPL(s, float, float)
BSVD_STRIDED_IMPL(d, double, double)
BSVD_STRIDED_IMPL(c, void, float)
BSVD_STRIDED_IMPL(z, void, double)

#define BSVD_BATCHED_IMPL(TAG, T, R)                                                          \
    bsvd_status bsvd_##TAG##gesvj_batched(BSVD_BATCHED_ARGS(T, R)) {                           \
        return batched_impl(#TAG[0], handle, jobu, jobv, batch, m, n,                          \
                            reinterpret_cast<const void* const*>(dA), lda,                     \
                            reinterpret_cast<void* const*>(dS),                                \
                            reinterpret_cast<void* const*>(dU), ldu,                           \
                            reinterpret_cast<void* const*>(dV), ldv, d_info, d_sweeps, d_work, \
                            work_bytes, opts, stream);                                         \
    }
BSVD_BATCHED_IMPL(s, float, float)
BSVD_BATCHED_IMPL(d, double, double)
BSVD_BATCHED_IMPL(c, void, float)
BSVD_BATCHED_IMPL(z, void, double)

}  // extern "C"
