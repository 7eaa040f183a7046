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
#include <tuple>
#include <utility>
#include <vector>

#include "bsvd.h"
#include "blocked_layout.h"
#include "gesvj_fused.cuh"
#include "internal.h"

// Autotuned choice for a bucket: (type, M and N rounded up to powers of two,
// jobu, jobv) -> path and block width.
struct bsvd_tuned {
    int path;
    int nb;
    float ms;
};
using bsvd_tune_key = std::tuple<char, int, int, int, int>;

struct bsvd_handle_s {
    int last_arg = 0;
    int last_cuda = 0;
    int device = -1;
    int max_smem = 0;      // opt-in shared memory per block (bytes)
    int sm_count = 0;
    std::map<bsvd_tune_key, bsvd_tuned> tuned;
    cudaStream_t cap = nullptr;   // private stream on which sweeps are recorded into CUDA graphs
    int cap_device = -1;
    cudaStream_t pipe[3] = {nullptr, nullptr, nullptr};   // host-buffer pipeline: H2D, D2H, 2nd compute
    int pipe_device = -1;
    cudaStream_t split = nullptr;                          // split uneven batches: the multi-kernel part
    cudaEvent_t split_ev[2] = {nullptr, nullptr};          // fork from, join to the caller's stream
    int split_device = -1;
    cudaStream_t pstream[5] = {};                          // persistent segments beyond the first
    cudaEvent_t pevent[5] = {};                            // their joins
    cudaEvent_t pfork = nullptr;                           // the fork from the caller's stream
    int pstream_device = -1, pstream_prio = 0;
};

namespace {

using bsvd::BlockedArgs;
using bsvd::FusedArgs;
using bsvd::blk_bytes;

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

// The stream on which the multi-kernel path records one sweep into a CUDA
// graph (never the caller's: the legacy default stream cannot be captured);
// nullptr when graphs are off (flags bit 3) or the stream cannot be made.
cudaStream_t capture_stream(bsvd_handle h, int flags) {
    if (flags & 8) return nullptr;
    if (h->cap && h->cap_device == h->device) return h->cap;
    if (h->cap) { cudaStreamDestroy(h->cap); h->cap = nullptr; }
    if (cudaStreamCreateWithFlags(&h->cap, cudaStreamNonBlocking) != cudaSuccess) {
        cudaGetLastError();
        h->cap = nullptr;
        return nullptr;
    }
    h->cap_device = h->device;
    return h->cap;
}

struct Resolved {
    int nb, max_sweeps, inner_sweeps, path, flags, prec;
    double tol;
};

// Options with defaults filled in.  Returns false for an invalid option.
bool resolve(const bsvd_opts* o, bool single, int N, Resolved& r) {
    bsvd_opts z;
    std::memset(&z, 0, sizeof z);
    if (!o) o = &z;
    if (o->nb < 0 || o->max_sweeps < 0 || o->inner_sweeps < 0 || o->tol < 0 || o->path < 0 ||
        o->path > BSVD_PATH_PERSISTENT || o->flags < 0 || o->flags > 8191 || o->prec < 0 ||
        o->prec > BSVD_PREC_MIXED || (o->prec == BSVD_PREC_MIXED && single))
        return false;
    r.nb = o->nb ? o->nb : (N >= 48 ? 16 : (N >= 12 ? 8 : 4));
    r.max_sweeps = o->max_sweeps ? o->max_sweeps : kDefaultMaxSweeps;
    r.max_sweeps = std::min(r.max_sweeps, bsvd::kMaxSweeps);
    r.path = o->path;
    r.inner_sweeps = o->inner_sweeps ? o->inner_sweeps : (r.path == BSVD_PATH_PLAIN ? 30 : 1);
    r.tol = o->tol > 0 ? o->tol : 30.0 * (single ? kU32 : kU64);
    r.flags = o->flags;
    r.prec = o->prec;
    return true;
}

int pow2_ceil(int x) {
    int p = 1;
    while (p < x) p <<= 1;
    return p;
}

bsvd_tune_key tune_key(char t, int m, int n, bool wantU, bool wantV) {
    return bsvd_tune_key(t, pow2_ceil(std::max(m, n)), pow2_ceil(std::min(m, n)), wantU ? 1 : 0, wantV ? 1 : 0);
}

// An AUTO call with no block width given follows the autotuned choice for its
// bucket, if bsvd_autotune recorded one in this handle.
void apply_tuned(bsvd_handle h, char t, int m, int n, bool wantU, bool wantV, const bsvd_opts* o,
                 Resolved& r) {
    if (!h || r.path != BSVD_PATH_AUTO || (o && o->nb) || r.prec != BSVD_PREC_NATIVE || (r.flags & 6)) return;
    auto it = h->tuned.find(tune_key(t, m, n, wantU, wantV));
    if (it == h->tuned.end()) return;
    r.path = it->second.path;
    r.nb = it->second.nb;
}

typedef size_t (*plan_fn)(int, int, int, bool, FusedArgs&, int&);
typedef cudaError_t (*launch_fn)(int, const FusedArgs&, int, size_t, cudaStream_t);
typedef cudaError_t (*blocked_fn)(int, const BlockedArgs&, void*, cudaStream_t, bool, bool, cudaStream_t);
typedef cudaError_t (*blocked_var_fn)(int, const BlockedArgs&, const bsvd::BlkVarPlan&, void*, cudaStream_t,
                                      cudaStream_t);
typedef cudaError_t (*persist_fn)(int, bool, size_t, const bsvd::PersistArgs&, int, int, cudaStream_t);
typedef long long (*slot_fn)(int, int, int);
typedef size_t (*psmem_fn)(int, size_t, int);

struct TypeOps {
    bool single;
    size_t elt;
    plan_fn plan;
    launch_fn launch;
    blocked_fn blocked;
    persist_fn persist;
    slot_fn slot;
    blocked_var_fn blocked_var;
    psmem_fn smem;
};

TypeOps ops_for(char t) {
    switch (t) {
        case 's': return {true, 4, bsvd::fused_plan_s, bsvd::fused_launch_s, bsvd::blocked_run_s,
                          bsvd::persist_launch_s, bsvd::persist_slot_s, bsvd::blocked_run_var_s,
                          bsvd::persist_smem_s};
        case 'd': return {false, 8, bsvd::fused_plan_d, bsvd::fused_launch_d, bsvd::blocked_run_d,
                          bsvd::persist_launch_d, bsvd::persist_slot_d, bsvd::blocked_run_var_d,
                          bsvd::persist_smem_d};
        case 'c': return {true, 8, bsvd::fused_plan_c, bsvd::fused_launch_c, bsvd::blocked_run_c,
                          bsvd::persist_launch_c, bsvd::persist_slot_c, bsvd::blocked_run_var_c,
                          bsvd::persist_smem_c};
        default:  return {false, 16, bsvd::fused_plan_z, bsvd::fused_launch_z, bsvd::blocked_run_z,
                          bsvd::persist_launch_z, bsvd::persist_slot_z, bsvd::blocked_run_var_z,
                          bsvd::persist_smem_z};
    }
}

// How one group of equal-shape matrices runs.
struct Plan {
    bool blocked = false;
    FusedArgs a;               // fused path
    size_t smem = 0;
    int threads = 0;
    int nb = 0;
    bool two_stage = false, masks = true, host_sync = false;
    bool mixed = false;        // FP64 output by the mixed-precision path (bytes: its workspace)
    size_t bytes = 0;          // workspace of the multi-kernel path
};

bool fused_nb(int nb) { return nb == 4 || nb == 8 || nb == 16; }
bool blocked_nb(int nb) { return nb == 4 || nb == 8 || nb == 16 || nb == 32; }

bsvd_status plan_group(int max_smem, const TypeOps& ops, int m, int n, int count, bool wantU,
                       bool wantV, const Resolved& r, Plan& p) {
    std::memset(&p.a, 0, sizeof p.a);
    const int M = std::max(m, n), N = std::min(m, n);
    const bool needVs = (m < n) ? wantU : wantV;
    p.nb = r.nb;
    p.blocked = false;
    const bool want_blocked_opts = (r.flags & 6) != 0;
    if (r.path == BSVD_PATH_FUSED || (r.path == BSVD_PATH_AUTO && !want_blocked_opts)) {
        if (fused_nb(r.nb)) {
            p.smem = ops.plan(r.nb, M, N, needVs, p.a, p.threads);
            if (p.smem > 0 && p.smem <= (size_t)max_smem) {
                FusedArgs& a = p.a;
                a.m = m; a.n = n; a.trans = m < n; a.M = M; a.N = N;
                a.wantU = wantU; a.wantV = wantV;
                a.tol = r.tol; a.max_sweeps = r.max_sweeps; a.inner_sweeps = r.inner_sweeps;
                a.flags = r.flags;
                return BSVD_OK;
            }
        }
        if (r.path == BSVD_PATH_FUSED) return BSVD_ERR_NOT_IMPLEMENTED;   // does not fit on chip
    }
    if (!blocked_nb(r.nb)) return BSVD_ERR_NOT_IMPLEMENTED;
    p.blocked = true;
    p.two_stage = r.path == BSVD_PATH_PLAIN || (r.flags & 2);
    p.masks = !(r.path == BSVD_PATH_PLAIN || (r.flags & 4));
    p.host_sync = !p.masks;
    p.bytes = bsvd::blocked_bytes(r.nb, M, N, count, p.two_stage, ops.elt);
    return BSVD_OK;
}

BlockedArgs blocked_args(int m, int n, int count, bool wantU, bool wantV, const Resolved& r, bool masks) {
    BlockedArgs a;
    std::memset(&a, 0, sizeof a);
    a.m = m; a.n = n; a.trans = m < n; a.M = std::max(m, n); a.N = std::min(m, n);
    a.count = count;
    a.wantU = wantU; a.wantV = wantV;
    a.tol = r.tol; a.max_sweeps = r.max_sweeps; a.inner_sweeps = r.inner_sweeps;
    a.flags = r.flags; a.masks = masks;
    return a;
}

size_t align256(size_t x) { return (x + 255) & ~size_t(255); }

// Workspace of the pointer-array form: lda, ldu, ldv (3 x batch ints) and the
// matrix ids grouped by shape (batch ints), then each multi-kernel group's
// region in shape order.
size_t batched_ints(int batch) { return align256((size_t)4 * batch * sizeof(int)); }

int device_smem_or_default(bsvd_handle h) {
    int dev = 0, v = 0;
    if (h->device >= 0) return h->max_smem;
    if (cudaGetDevice(&dev) == cudaSuccess &&
        cudaDeviceGetAttribute(&v, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev) == cudaSuccess)
        return v;
    cudaGetLastError();
    return 232448;   // GB300: 227 KB opt-in shared memory per block
}

// ---- mixed precision (FP64 output from FP32 sweeps + FP64 polish) ----------
struct MixedPlan {
    Plan p32, p64;
    Resolved r32, r64;
    size_t off[8];        // A32, V32, S32, info32, V64, Vtmp, E, Ahat
    size_t off32, off64;  // workspace of the two solves (multi-kernel paths)
    size_t bytes;
};

bsvd_status plan_mixed(int max_smem, char t, int m, int n, int batch, bool wantU, bool wantV,
                       const Resolved& r, MixedPlan& mp) {
    const int M = std::max(m, n), N = std::min(m, n);
    const TypeOps o32 = ops_for(t == 'd' ? 's' : 'c'), o64 = ops_for(t);
    const bool trans = m < n;
    mp.r32 = r;
    mp.r32.tol = 30.0 * kU32;
    mp.r32.path = BSVD_PATH_AUTO;
    // FP32 sweeps: FMA tiles / FP64 rotations, and how the sweep loop runs
    // (no graph, host checks, host-replayed graph), as the caller asked
    mp.r32.flags = r.flags & (128 | 256 | 8 | 16 | 2048 | 4096);
    mp.r32.inner_sweeps = 1;
    mp.r32.prec = BSVD_PREC_NATIVE;
    mp.r64 = r;
    mp.r64.prec = BSVD_PREC_NATIVE;
    // FP32 solve: V only, on the working-orientation copy (M x N)
    bsvd_status st = plan_group(max_smem, o32, M, N, batch, false, true, mp.r32, mp.p32);
    if (st != BSVD_OK) return st;
    // FP64 polish on A_hat (M x N); its U/V are the caller's U/V, swapped for m < n
    const bool pu = trans ? wantV : wantU, pv = trans ? wantU : wantV;
    st = plan_group(max_smem, o64, M, N, batch, pu, pv, mp.r64, mp.p64);
    if (st != BSVD_OK) return st;
    const size_t b = (size_t)batch, mn = (size_t)M * N, nn = (size_t)N * N;
    const size_t sizes[8] = {b * mn * o32.elt, b * nn * o32.elt, b * N * 4, b * 2 * sizeof(int),
                             b * nn * o64.elt, b * nn * o64.elt, b * nn * o64.elt, b * mn * o64.elt};
    size_t pos = 0;
    for (int i = 0; i < 8; ++i) { mp.off[i] = pos; pos += align256(sizes[i]); }
    mp.off32 = pos;
    if (mp.p32.blocked) pos += align256(mp.p32.bytes);
    mp.off64 = pos;
    if (mp.p64.blocked) pos += align256(mp.p64.bytes);
    mp.bytes = pos;
    return BSVD_OK;
}

// Pointer-array inputs and outputs of one shape group of a pointer-array
// batch (device arrays indexed by matrix id; `index` lists the group's ids).
struct PtrIO {
    const void* const* Ap; const int* ldap;
    void* const* Sp;
    void* const* Up; const int* ldup;
    void* const* Vp; const int* ldvp;
    const int* index;
};

bsvd_status mixed_impl(char t, bsvd_handle h, bool wantU, bool wantV, int batch, int m, int n,
                       const void* dA, int lda, long long sA, void* dS, long long sS, void* dU,
                       int ldu, long long sU, void* dV, int ldv, long long sV, int* d_info,
                       int* d_sweeps, void* d_work, size_t work_bytes, const Resolved& r,
                       cudaStream_t s, const PtrIO* io = nullptr) {
    MixedPlan mp;
    bsvd_status st = plan_mixed(h->max_smem, t, m, n, batch, wantU, wantV, r, mp);
    if (st != BSVD_OK) return st;
    if (!d_work || work_bytes < mp.bytes) return BSVD_ERR_WORKSPACE;
    const int M = std::max(m, n), N = std::min(m, n);
    const bool trans = m < n;
    char* w = static_cast<char*>(d_work);
    bsvd::MixedArgs ma;
    ma.m = m; ma.n = n; ma.M = M; ma.N = N; ma.trans = trans;
    ma.A = dA; ma.sA = sA; ma.lda = lda;
    ma.Ap = io ? io->Ap : nullptr; ma.ldap = io ? io->ldap : nullptr; ma.index = io ? io->index : nullptr;
    ma.A32 = w + mp.off[0]; ma.V32 = w + mp.off[1];
    ma.V64 = w + mp.off[4]; ma.Vtmp = w + mp.off[5]; ma.E = w + mp.off[6]; ma.Ahat = w + mp.off[7];
    void* S32 = w + mp.off[2];
    int* info32 = reinterpret_cast<int*>(w + mp.off[3]);
    int* sweeps32 = info32 + batch;
    const TypeOps o32 = ops_for(t == 'd' ? 's' : 'c'), o64 = ops_for(t);
    cudaError_t e = (t == 'd') ? bsvd::mixed_prepare_d(ma, batch, s) : bsvd::mixed_prepare_z(ma, batch, s);
    if (e != cudaSuccess) return fail_cuda(h, e);
    // 1. FP32 solve for V32 (N x N, ld N)
    if (mp.p32.blocked) {
        BlockedArgs a = blocked_args(M, N, batch, false, true, mp.r32, mp.p32.masks);
        a.A = ma.A32; a.sA = (long long)M * N; a.lda = M;
        a.S = S32; a.sS = N;
        a.V = ma.V32; a.sV = (long long)N * N; a.ldv = N;
        a.info = info32; a.sweeps = sweeps32;
        e = o32.blocked(mp.p32.nb, a, w + mp.off32, s, mp.p32.two_stage, mp.p32.host_sync, capture_stream(h, r.flags));
    } else {
        FusedArgs& a = mp.p32.a;
        a.A = ma.A32; a.sA = (long long)M * N; a.lda = M;
        a.S = S32; a.sS = N;
        a.V = ma.V32; a.sV = (long long)N * N; a.ldv = N;
        a.info = info32; a.sweeps = sweeps32;
        e = o32.launch(mp.p32.nb, a, batch, mp.p32.smem, s);
    }
    if (e != cudaSuccess) return fail_cuda(h, e);
    // 2. orthonormal V in FP64 and A_hat = A V
    e = (t == 'd') ? bsvd::mixed_restore_d(ma, batch, s) : bsvd::mixed_restore_z(ma, batch, s);
    if (e != cudaSuccess) return fail_cuda(h, e);
    // 3. FP64 polish on A_hat from V64; outputs go straight to the caller (U and V
    //    swap roles for m < n: A^H = V Sigma U^H)
    void* pU = trans ? dV : dU;
    void* pV = trans ? dU : dV;
    const int pldu = trans ? ldv : ldu, pldv = trans ? ldu : ldv;
    const long long psU = trans ? sV : sU, psV = trans ? sU : sV;
    const bool pu = trans ? wantV : wantU, pv = trans ? wantU : wantV;
    // pointer-array outputs: by matrix id, the strided A_hat and V64 by
    // position in the group (in_local)
    auto outputs = [&](auto& a) {
        if (!io) return;
        a.S = nullptr; a.U = nullptr; a.V = nullptr;
        a.Sp = io->Sp;
        a.Up = trans ? io->Vp : io->Up; a.ldup = trans ? io->ldvp : io->ldup;
        a.Vp = trans ? io->Up : io->Vp; a.ldvp = trans ? io->ldup : io->ldvp;
        a.index = io->index;
        a.in_local = 1;
    };
    if (mp.p64.blocked) {
        BlockedArgs a = blocked_args(M, N, batch, pu, pv, mp.r64, mp.p64.masks);
        a.A = ma.Ahat; a.sA = (long long)M * N; a.lda = M;
        a.V0 = pv ? ma.V64 : nullptr; a.sV0 = (long long)N * N; a.ldv0 = N;
        a.S = dS; a.sS = sS;
        a.U = pU; a.sU = psU; a.ldu = pldu;
        a.V = pV; a.sV = psV; a.ldv = pldv;
        a.info = d_info; a.sweeps = d_sweeps;
        outputs(a);
        e = o64.blocked(mp.p64.nb, a, w + mp.off64, s, mp.p64.two_stage, mp.p64.host_sync, capture_stream(h, r.flags));
    } else {
        FusedArgs& a = mp.p64.a;
        a.A = ma.Ahat; a.sA = (long long)M * N; a.lda = M;
        a.V0 = pv ? ma.V64 : nullptr; a.sV0 = (long long)N * N; a.ldv0 = N;
        a.S = dS; a.sS = sS;
        a.U = pU; a.sU = psU; a.ldu = pldu;
        a.V = pV; a.sV = psV; a.ldv = pldv;
        a.info = d_info; a.sweeps = d_sweeps;
        outputs(a);
        e = o64.launch(mp.p64.nb, a, batch, mp.p64.smem, s);
    }
    return e == cudaSuccess ? BSVD_OK : fail_cuda(h, e);
}

// ---- QR pre-processing (flags bit 5) ----------------------------------------
constexpr int kFlagQR = 32;

struct QrPlan {
    Plan p;              // the SVD of R (N x N)
    Resolved r;
    size_t off[5];       // W, tau, R, ex, Uhat
    size_t offp;         // the R-SVD's multi-kernel workspace
    size_t bytes;
};

bsvd_status plan_qr(int max_smem, const TypeOps& ops, int m, int n, int batch, bool wantU, bool wantV,
                    const Resolved& r, QrPlan& qp) {
    const int M = std::max(m, n), N = std::min(m, n);
    const bool trans = m < n;
    const bool wy = trans ? wantV : wantU, wv = trans ? wantU : wantV;   // Q side, R's right side
    qp.r = r;
    qp.r.flags &= ~kFlagQR;
    bsvd_status st = plan_group(max_smem, ops, N, N, batch, wy, wv, qp.r, qp.p);
    if (st != BSVD_OK) return st;
    const size_t b = (size_t)batch, e = ops.elt;
    const size_t sizes[5] = {b * M * N * e, b * N * e, b * N * N * e, b * sizeof(int), wy ? b * N * N * e : 0};
    size_t pos = 0;
    for (int i = 0; i < 5; ++i) { qp.off[i] = pos; pos += align256(sizes[i]); }
    qp.offp = pos;
    if (qp.p.blocked) pos += align256(qp.p.bytes);
    qp.bytes = pos;
    return BSVD_OK;
}

// A' = Q [R; 0] (A' = A, or A^H when m < n), R = U_R Sigma V_R^H by the regular
// paths, then the left vectors of A' are Q [U_R; 0] and its right ones V_R.
bsvd_status qr_impl(char t, bsvd_handle h, bool wantU, bool wantV, int batch, int m, int n, const void* dA,
                    int lda, long long sA, void* dS, long long sS, void* dU, int ldu, long long sU, void* dV,
                    int ldv, long long sV, int* d_info, int* d_sweeps, void* d_work, size_t work_bytes,
                    const Resolved& r, cudaStream_t s) {
    const TypeOps ops = ops_for(t);
    QrPlan qp;
    bsvd_status st = plan_qr(h->max_smem, ops, m, n, batch, wantU, wantV, r, qp);
    if (st != BSVD_OK) return st;
    if (!d_work || work_bytes < qp.bytes) return BSVD_ERR_WORKSPACE;
    const int M = std::max(m, n), N = std::min(m, n);
    const bool trans = m < n;
    const bool wy = trans ? wantV : wantU, wv = trans ? wantU : wantV;
    char* w = static_cast<char*>(d_work);
    bsvd::QrArgs qa;
    std::memset(&qa, 0, sizeof qa);
    qa.m = m; qa.n = n; qa.M = M; qa.N = N; qa.trans = trans;
    qa.A = dA; qa.sA = sA; qa.lda = lda;
    qa.W = w + qp.off[0]; qa.tau = w + qp.off[1]; qa.R = w + qp.off[2];
    qa.ex = reinterpret_cast<int*>(w + qp.off[3]);
    qa.Uhat = wy ? w + qp.off[4] : nullptr;
    qa.Y = wy ? (trans ? dV : dU) : nullptr;
    qa.sY = trans ? sV : sU;
    qa.ldy = trans ? ldv : ldu;
    qa.S = dS; qa.sS = sS;
    cudaError_t e;
    switch (t) {
        case 's': e = bsvd::qr_factor_s(qa, batch, s); break;
        case 'd': e = bsvd::qr_factor_d(qa, batch, s); break;
        case 'c': e = bsvd::qr_factor_c(qa, batch, s); break;
        default:  e = bsvd::qr_factor_z(qa, batch, s); break;
    }
    if (e != cudaSuccess) return fail_cuda(h, e);
    // the SVD of R: its U to the workspace, its V straight to the caller
    void* pV = trans ? dU : dV;
    const int pldv = trans ? ldu : ldv;
    const long long psV = trans ? sU : sV;
    if (qp.p.blocked) {
        BlockedArgs a = blocked_args(N, N, batch, wy, wv, qp.r, qp.p.masks);
        a.A = qa.R; a.sA = (long long)N * N; a.lda = N;
        a.S = dS; a.sS = sS;
        a.U = qa.Uhat; a.sU = (long long)N * N; a.ldu = N;
        a.V = pV; a.sV = psV; a.ldv = pldv;
        a.info = d_info; a.sweeps = d_sweeps;
        e = ops.blocked(qp.p.nb, a, w + qp.offp, s, qp.p.two_stage, qp.p.host_sync, capture_stream(h, qp.r.flags));
    } else {
        FusedArgs& a = qp.p.a;
        a.A = qa.R; a.sA = (long long)N * N; a.lda = N;
        a.S = dS; a.sS = sS;
        a.U = qa.Uhat; a.sU = (long long)N * N; a.ldu = N;
        a.V = pV; a.sV = psV; a.ldv = pldv;
        a.info = d_info; a.sweeps = d_sweeps;
        e = ops.launch(qp.p.nb, a, batch, qp.p.smem, s);
    }
    if (e != cudaSuccess) return fail_cuda(h, e);
    switch (t) {
        case 's': e = bsvd::qr_apply_s(qa, batch, s); break;
        case 'd': e = bsvd::qr_apply_d(qa, batch, s); break;
        case 'c': e = bsvd::qr_apply_c(qa, batch, s); break;
        default:  e = bsvd::qr_apply_z(qa, batch, s); break;
    }
    return e == cudaSuccess ? BSVD_OK : fail_cuda(h, e);
}

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
    if (d_work && (reinterpret_cast<uintptr_t>(d_work) & 15) != 0) return fail_arg(h, 20);
    const TypeOps ops = ops_for(t);
    Resolved r;
    if (!resolve(opts, ops.single, k, r)) return fail_arg(h, 22);
    if (r.path == BSVD_PATH_PERSISTENT) r.path = BSVD_PATH_AUTO;   // one shape: the regular paths
    apply_tuned(h, t, m, n, wantU, wantV, opts, r);
    if (batch == 0) return BSVD_OK;
    bsvd_status st = refresh_device(h);
    if (st != BSVD_OK) return st;
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    if (k == 0) {   // empty matrices: nothing to compute, converged by definition
        cudaError_t e = cudaMemsetAsync(d_info, 0, sizeof(int) * (size_t)batch, s);
        if (e == cudaSuccess && d_sweeps) e = cudaMemsetAsync(d_sweeps, 0, sizeof(int) * (size_t)batch, s);
        return e == cudaSuccess ? BSVD_OK : fail_cuda(h, e);
    }
    if (r.flags & kFlagQR) {
        if (r.prec == BSVD_PREC_MIXED) return BSVD_ERR_NOT_IMPLEMENTED;
        return qr_impl(t, h, wantU, wantV, batch, m, n, dA, lda, sA, dS, sS, dU, ldu, sU, dV, ldv, sV, d_info,
                       d_sweeps, d_work, work_bytes, r, s);
    }
    if (r.prec == BSVD_PREC_MIXED)
        return mixed_impl(t, h, wantU, wantV, batch, m, n, dA, lda, sA, dS, sS, dU, ldu, sU, dV,
                          ldv, sV, d_info, d_sweeps, d_work, work_bytes, r, s);
    Plan p;
    st = plan_group(h->max_smem, ops, m, n, batch, wantU, wantV, r, p);
    if (st != BSVD_OK) return st;
    if (p.blocked) {
        if (!d_work || work_bytes < p.bytes) return BSVD_ERR_WORKSPACE;
        BlockedArgs a = blocked_args(m, n, batch, wantU, wantV, r, p.masks);
        a.A = dA; a.sA = sA; a.lda = lda;
        a.S = dS; a.sS = sS;
        a.U = dU; a.sU = sU; a.ldu = ldu;
        a.V = dV; a.sV = sV; a.ldv = ldv;
        a.info = d_info;
        a.sweeps = d_sweeps;
        cudaError_t e = ops.blocked(p.nb, a, d_work, s, p.two_stage, p.host_sync, capture_stream(h, r.flags));
        return e == cudaSuccess ? BSVD_OK : fail_cuda(h, e);
    }
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

// Shape groups of a pointer-array batch, in a fixed order.
using Groups = std::map<std::pair<int, int>, std::vector<int>>;

bsvd_status plan_batched(bsvd_handle h, char t, int max_smem, const TypeOps& ops, int batch,
                         const Groups& groups, bool wantU, bool wantV, const bsvd_opts* opts,
                         std::vector<Plan>& plans, std::vector<Resolved>& res, size_t& total) {
    total = batched_ints(batch);
    plans.assign(groups.size(), Plan());
    res.assign(groups.size(), Resolved());
    size_t gi = 0;
    for (auto& kv : groups) {
        const int mm = kv.first.first, nn = kv.first.second;
        if (!resolve(opts, ops.single, std::min(mm, nn), res[gi])) return BSVD_ERR_INVALID;
        apply_tuned(h, t, mm, nn, wantU, wantV, opts, res[gi]);
        if (std::min(mm, nn) > 0 && res[gi].prec == BSVD_PREC_MIXED) {
            MixedPlan mp;
            bsvd_status st = plan_mixed(max_smem, t, mm, nn, (int)kv.second.size(), wantU, wantV, res[gi], mp);
            if (st != BSVD_OK) return st;
            plans[gi].mixed = true;
            plans[gi].bytes = mp.bytes;
            total += align256(mp.bytes);
        } else if (std::min(mm, nn) > 0) {
            bsvd_status st = plan_group(max_smem, ops, mm, nn, (int)kv.second.size(), wantU, wantV,
                                        res[gi], plans[gi]);
            if (st != BSVD_OK) return st;
            if (plans[gi].blocked) total += align256(plans[gi].bytes);
        }
        ++gi;
    }
    return BSVD_OK;
}

// ---- persistent launches for a pointer-array batch of any shapes -------------
// The batch is cut into segments, one per (block width, where the working
// arrays live): each matrix gets the block width of its own shape -- the
// caller's nb, else the autotuned choice recorded in the handle for its
// bucket (type, M and N rounded up to powers of two, jobs), else the AUTO
// rule from min(m, n) -- and runs with W and V in shared memory when they
// fit there at the kernel's occupancy (the on-chip kernel's layout), else in
// a global-memory slot of its CTA.  Each segment is one persistent launch
// whose CTAs take its matrices largest first; the segments run on streams
// forked from the caller's (the largest segment on the caller's own), so a
// later segment's CTAs fill the SMs that an earlier one's tail leaves idle.
constexpr int kMaxPersistSegs = 6;
constexpr int kFlagNoOnChip = 512;   // flags bit 9: every matrix in a global slot

struct PersistSeg {
    int nb = 0;
    bool onchip = false;
    std::vector<int> ids;          // largest first
    int grid = 0, maxN = 0;
    long long slot = 0;            // elements per global slot
    size_t wv = 0;                 // bytes of W + V of the segment's largest matrix on chip
    size_t ws_off = 0;             // byte offset of the segment's slots in the workspace
    double work = 0;               // sum of M N^2
};

struct PersistPlan {
    std::vector<PersistSeg> segs;
    std::vector<int> nb_of, where_of;   // per matrix: block width; 0 slot, 1 on chip, -1 not here
    int count = 0, maxN = 0;
    size_t ints = 0, bytes = 0;
};

int device_sms_or_default(bsvd_handle h) {
    int dev = 0, v = 0;
    if (h->device >= 0) return h->sm_count;
    if (cudaGetDevice(&dev) == cudaSuccess &&
        cudaDeviceGetAttribute(&v, cudaDevAttrMultiProcessorCount, dev) == cudaSuccess)
        return v;
    cudaGetLastError();
    return 152;   // GB300
}

// Block width of one matrix of a persistent batch.
int persist_nb(bsvd_handle h, char t, int m, int n, bool wantU, bool wantV, const bsvd_opts* opts) {
    if (opts && opts->nb) return opts->nb;
    if (h) {
        auto it = h->tuned.find(tune_key(t, m, n, wantU, wantV));
        if (it != h->tuned.end() && fused_nb(it->second.nb)) return it->second.nb;
    }
    const int k = std::min(m, n);
    return k >= 48 ? 16 : (k >= 12 ? 8 : 4);
}

// Shared memory one CTA of an on-chip launch may take: half the SM's 228 KB
// less the 1 KB the hardware reserves per CTA, so that at least two CTAs
// share an SM -- a CTA that filled the SM would hold it alone for its whole
// matrix, and no other launch's CTA could start there meanwhile.
size_t onchip_budget(const TypeOps& ops, int max_smem) {
    (void)ops;
    return std::min((size_t)(228 * 1024 / 2 - 1024), (size_t)max_smem);
}

bsvd_status plan_persistent(bsvd_handle h, char t, int sms, int max_smem, const TypeOps& ops, int batch,
                            const int* m, const int* n, bool wantU, bool wantV, const bsvd_opts* opts,
                            PersistPlan& pp, const std::vector<char>* excl = nullptr) {
    pp = PersistPlan();
    pp.nb_of.assign(batch, 0);
    pp.where_of.assign(batch, -1);
    std::vector<int> ids;
    for (int i = 0; i < batch; ++i) {
        if (excl && (*excl)[i]) continue;             // solved on the multi-kernel path
        const int k = std::min(m[i], n[i]);
        if (k > 0) ids.push_back(i);
        pp.maxN = std::max(pp.maxN, k);
    }
    // largest first: cost ~ M N^2 per sweep
    auto cost = [&](int i) { return (double)std::max(m[i], n[i]) * std::min(m[i], n[i]) * std::min(m[i], n[i]); };
    std::stable_sort(ids.begin(), ids.end(), [&](int a, int b) { return cost(a) > cost(b); });
    pp.count = (int)ids.size();
    const bool allow_onchip = !(opts && (opts->flags & kFlagNoOnChip));
    const size_t budget = onchip_budget(ops, max_smem);
    std::map<std::pair<int, int>, int> seg_of;         // (nb, on chip) -> segment
    for (int id : ids) {
        const int nb = persist_nb(h, t, m[id], n[id], wantU, wantV, opts);
        if (!fused_nb(nb)) return BSVD_ERR_NOT_IMPLEMENTED;
        const size_t wv = ops.slot(nb, m[id], n[id]) * ops.elt;
        const bool onchip = allow_onchip && ops.smem(nb, wv, pp.maxN) <= budget;
        auto key = std::make_pair(nb, onchip ? 1 : 0);
        auto it = seg_of.find(key);
        if (it == seg_of.end()) {
            it = seg_of.emplace(key, (int)pp.segs.size()).first;
            pp.segs.emplace_back();
            pp.segs.back().nb = nb;
            pp.segs.back().onchip = onchip;
        }
        PersistSeg& sg = pp.segs[it->second];
        sg.ids.push_back(id);
        sg.maxN = std::max(sg.maxN, std::min(m[id], n[id]));
        if (onchip) sg.wv = std::max(sg.wv, wv);
        else sg.slot = std::max(sg.slot, ops.slot(nb, m[id], n[id]));
        sg.work += cost(id);
        pp.nb_of[id] = nb;
        pp.where_of[id] = onchip ? 1 : 0;
    }
    std::stable_sort(pp.segs.begin(), pp.segs.end(),
                     [](const PersistSeg& a, const PersistSeg& b) { return a.work > b.work; });
    if ((int)pp.segs.size() > kMaxPersistSegs) return BSVD_ERR_NOT_IMPLEMENTED;
    // ints: lda, ldu, ldv, m, n (batch each), the segments' queues (count in
    // all), one queue head per segment
    pp.ints = align256(((size_t)5 * batch + pp.count + kMaxPersistSegs) * sizeof(int));
    size_t pos = pp.ints;
    for (PersistSeg& sg : pp.segs) {
        // global slots: two resident CTAs per SM (register cap 128) except
        // for complex128, and that many slots; on chip the launch sizes the
        // grid by the kernel's occupancy, capped here by the matrix count
        const int per_sm = (ops.elt == 16 ? 1 : 2) * (16 / sg.nb);   // 256 threads' worth of CTAs, x2
        sg.grid = sg.onchip ? std::max(1, (int)sg.ids.size())
                            : std::max(1, std::min((int)sg.ids.size(), sms * per_sm));
        sg.ws_off = pos;
        if (!sg.onchip) pos += align256((size_t)sg.grid * sg.slot * ops.elt);
    }
    pp.bytes = pos;
    return BSVD_OK;
}

// The side streams of the persistent segments, with the priority of the
// caller's stream `s` (the server runs small requests on high-priority
// streams): made once per device and priority.
cudaError_t persist_streams(bsvd_handle h, cudaStream_t s) {
    int prio = 0;
    cudaError_t e = cudaStreamGetPriority(s, &prio);
    if (e != cudaSuccess) return e;
    if (h->pstream[0] && h->pstream_device == h->device && h->pstream_prio == prio) return cudaSuccess;
    for (int i = 0; i < kMaxPersistSegs - 1; ++i) {
        if (h->pstream[i]) cudaStreamDestroy(h->pstream[i]);
        if (h->pevent[i]) cudaEventDestroy(h->pevent[i]);
        h->pstream[i] = nullptr;
        h->pevent[i] = nullptr;
    }
    if (h->pfork) cudaEventDestroy(h->pfork);
    h->pfork = nullptr;
    e = cudaEventCreateWithFlags(&h->pfork, cudaEventDisableTiming);
    for (int i = 0; i < kMaxPersistSegs - 1 && e == cudaSuccess; ++i) {
        e = cudaStreamCreateWithPriority(&h->pstream[i], cudaStreamNonBlocking, prio);
        if (e == cudaSuccess) e = cudaEventCreateWithFlags(&h->pevent[i], cudaEventDisableTiming);
    }
    if (e == cudaSuccess) {
        h->pstream_device = h->device;
        h->pstream_prio = prio;
    }
    return e;
}

bsvd_status persistent_impl(bsvd_handle h, char t, const TypeOps& ops, bool wantU, bool wantV, int batch,
                            const int* m, const int* n, const void* const* dA, const int* lda,
                            void* const* dS, void* const* dU, const int* ldu, void* const* dV,
                            const int* ldv, int* d_info, int* d_sweeps, void* d_work,
                            size_t work_bytes, const bsvd_opts* opts, cudaStream_t s, int* d_done = nullptr,
                            const int* d_abort = nullptr, const std::vector<char>* excl = nullptr) {
    PersistPlan pp;
    bsvd_status st = plan_persistent(h, t, h->sm_count, h->max_smem, ops, batch, m, n, wantU, wantV, opts, pp, excl);
    if (st != BSVD_OK) return st;
    if (!d_work || work_bytes < pp.bytes) return BSVD_ERR_WORKSPACE;
    Resolved r;
    if (!resolve(opts, ops.single, pp.maxN, r)) return fail_arg(h, 18);
    // ints: lda, ldu, ldv, m, n (batch each), the queues, the heads (zero)
    std::vector<int> host((size_t)5 * batch + pp.count + kMaxPersistSegs, 0);
    for (int i = 0; i < batch; ++i) {
        host[i] = lda[i];
        host[batch + i] = wantU ? ldu[i] : 1;
        host[2 * (size_t)batch + i] = wantV ? ldv[i] : 1;
        host[3 * (size_t)batch + i] = m[i];
        host[4 * (size_t)batch + i] = n[i];
    }
    std::vector<size_t> qpos;
    size_t q = 5 * (size_t)batch;
    for (const PersistSeg& sg : pp.segs) {
        qpos.push_back(q);
        std::copy(sg.ids.begin(), sg.ids.end(), host.begin() + q);
        q += sg.ids.size();
    }
    int* dws = static_cast<int*>(d_work);
    cudaError_t e = cudaMemcpyAsync(dws, host.data(), sizeof(int) * host.size(), cudaMemcpyHostToDevice, s);
    if (e != cudaSuccess) return fail_cuda(h, e);
    for (int i = 0; i < batch; ++i)
        if (std::min(m[i], n[i]) == 0) {
            e = cudaMemsetAsync(d_info + i, 0, sizeof(int), s);
            if (e == cudaSuccess && d_sweeps) e = cudaMemsetAsync(d_sweeps + i, 0, sizeof(int), s);
            if (e != cudaSuccess) return fail_cuda(h, e);
        }
    if (pp.count == 0) return BSVD_OK;
    const int nseg = (int)pp.segs.size();
    if (nseg > 1) {
        if ((e = persist_streams(h, s)) != cudaSuccess) return fail_cuda(h, e);
        if ((e = cudaEventRecord(h->pfork, s)) != cudaSuccess) return fail_cuda(h, e);
    }
    cudaError_t first_err = cudaSuccess;
    for (int k = 0; k < nseg; ++k) {
        const PersistSeg& sg = pp.segs[k];
        cudaStream_t ss = k == 0 ? s : h->pstream[k - 1];
        if (k > 0 && (e = cudaStreamWaitEvent(ss, h->pfork, 0)) != cudaSuccess) {
            first_err = e;
            break;
        }
        bsvd::PersistArgs p;
        std::memset(&p, 0, sizeof p);
        FusedArgs& a = p.base;
        a.Ap = dA; a.ldap = dws;
        a.Sp = dS;
        a.Up = dU; a.ldup = dws + batch;
        a.Vp = dV; a.ldvp = dws + 2 * batch;
        a.info = d_info; a.sweeps = d_sweeps;
        a.wantU = wantU; a.wantV = wantV;
        a.tol = r.tol; a.max_sweeps = r.max_sweeps; a.inner_sweeps = r.inner_sweeps; a.flags = r.flags;
        p.mm = dws + 3 * batch;
        p.nn = dws + 4 * batch;
        p.order = dws + qpos[k];
        p.count = (int)sg.ids.size();
        p.head = dws + 5 * batch + pp.count + k;
        p.ws = static_cast<char*>(d_work) + sg.ws_off;
        p.slot_elems = sg.slot;
        p.done = d_done;
        p.abort = d_abort;
        e = ops.persist(sg.nb, sg.onchip, sg.wv, p, sg.grid, sg.maxN, ss);
        if (e != cudaSuccess) {
            first_err = e;
            break;
        }
    }
    // join every side stream that was forked, also after a failure: the
    // caller's stream owns the results
    if (nseg > 1)
        for (int k = 1; k < nseg; ++k) {
            cudaError_t ej = cudaEventRecord(h->pevent[k - 1], h->pstream[k - 1]);
            if (ej == cudaSuccess) ej = cudaStreamWaitEvent(s, h->pevent[k - 1], 0);
            if (first_err == cudaSuccess) first_err = ej;
        }
    return first_err == cudaSuccess ? BSVD_OK : fail_cuda(h, first_err);
}

// ---- flags bit 6: split an uneven complex64 persistent batch ------------------
// Matrices with min(m, n) >= split_k run on the multi-kernel path as one
// variable-shape batch (per-matrix shapes, CUDA-graph sweeps) on a stream of
// the handle, beside the persistent launch for the rest.  With W in global
// memory the persistent kernel's inner solver runs four block pairs per SM;
// the multi-kernel path runs every pair of every large matrix at once.
// Measured on the uneven workload's 4,224 complex64 matrices with k >= 128:
// 2.47 s against 3.11 s in the persistent launch (with flags bit 4; without
// it the empty sweeps up to max_sweeps cost 0.3 s).  For FP32 the
// variable-shape batch was slower (1.31 s against 1.20 s), so the flag
// leaves other types in the persistent launch.
// Flags bit 10 extends the split to real FP32 (measured on the uneven
// workload; the default leaves FP32 in the persistent launches).  The split
// starts at min(m, n) >= 112 for complex64 and 144 for FP32: batches of 600
// matrices m ~ U{n..2n} took (persistent launch against split, ms) complex64
// 24.8 / 24.6 at n = 96, 33.9 / 29.3 at 112; FP32 21.3 / 22.9 at 112,
// 23.7 / 25.4 at 128, 31.7 / 30.1 at 144.
constexpr int kFlagSplit = 64, kFlagSplitF32 = 1024;
int split_k(const TypeOps& ops) { return ops.elt == 8 ? 112 : 144; }

bool split_large(const TypeOps& ops, const bsvd_opts* opts) {
    if (!ops.single || !opts || opts->path != BSVD_PATH_PERSISTENT || !(opts->flags & kFlagSplit)) return false;
    return ops.elt == 8 || (opts->flags & kFlagSplitF32);
}

struct SplitPlan {
    std::vector<char> excl;        // by matrix id: on the multi-kernel path
    std::vector<int> ids;          // those ids, in order
    bsvd::BlkVarPlan var;
    int nb = 16;
    size_t ints = 0, bytes = 0;    // ids + lda, ldu, ldv (batch each); then the multi-kernel workspace
};

void plan_split(const TypeOps& ops, int batch, const int* m, const int* n, const bsvd_opts* opts, SplitPlan& sp) {
    sp.excl.assign(batch, 0);
    sp.ids.clear();
    std::vector<int> mm, nn;
    const int k_split = split_k(ops);
    for (int i = 0; i < batch; ++i)
        if (std::min(m[i], n[i]) >= k_split) {
            sp.excl[i] = 1;
            sp.ids.push_back(i);
            mm.push_back(m[i]);
            nn.push_back(n[i]);
        }
    sp.nb = (opts && opts->nb) ? opts->nb : 16;
    const int count = (int)sp.ids.size();
    bsvd::blk_var_plan(sp.nb, count, mm.data(), nn.data(), ops.elt, sp.var);
    sp.ints = align256(((size_t)count + 3 * (size_t)batch) * sizeof(int));
    sp.bytes = count ? sp.ints + align256(sp.var.bytes) : 0;
}

cudaError_t split_streams(bsvd_handle h) {
    if (h->split && h->split_device == h->device) return cudaSuccess;
    if (h->split) cudaStreamDestroy(h->split);
    for (cudaEvent_t& ev : h->split_ev)
        if (ev) cudaEventDestroy(ev);
    h->split = nullptr;
    h->split_ev[0] = h->split_ev[1] = nullptr;
    cudaError_t e = cudaStreamCreateWithFlags(&h->split, cudaStreamNonBlocking);
    for (cudaEvent_t& ev : h->split_ev)
        if (e == cudaSuccess) e = cudaEventCreateWithFlags(&ev, cudaEventDisableTiming);
    if (e == cudaSuccess) h->split_device = h->device;
    return e;
}

bsvd_status split_impl(bsvd_handle h, char t, const TypeOps& ops, bool wantU, bool wantV, int batch, const int* m,
                       const int* n, const void* const* dA, const int* lda, void* const* dS, void* const* dU,
                       const int* ldu, void* const* dV, const int* ldv, int* d_info, int* d_sweeps,
                       void* d_work, size_t work_bytes, const bsvd_opts* opts, cudaStream_t s) {
    SplitPlan sp;
    plan_split(ops, batch, m, n, opts, sp);
    PersistPlan pp;
    bsvd_status st = plan_persistent(h, t, h->sm_count, h->max_smem, ops, batch, m, n, wantU, wantV, opts, pp,
                                     &sp.excl);
    if (st != BSVD_OK) return st;
    if (!d_work || work_bytes < pp.bytes + sp.bytes) return BSVD_ERR_WORKSPACE;
    const int count = (int)sp.ids.size();
    Resolved r;
    if (count > 0 && !resolve(opts, ops.single, sp.var.Nmax, r)) return fail_arg(h, 18);
    cudaError_t e = cudaSuccess;
    if (count > 0) {
        if ((e = split_streams(h)) != cudaSuccess) return fail_cuda(h, e);
        // fork: the side stream starts after the work already queued on the caller's
        if ((e = cudaEventRecord(h->split_ev[0], s)) != cudaSuccess) return fail_cuda(h, e);
    }
    // the persistent launch first: with flags bit 4 the multi-kernel part
    // below returns only once its matrices have converged
    st = persistent_impl(h, t, ops, wantU, wantV, batch, m, n, dA, lda, dS, dU, ldu, dV, ldv, d_info, d_sweeps,
                         d_work, pp.bytes, opts, s, nullptr, nullptr, &sp.excl);
    if (st != BSVD_OK || count == 0) return st;
    cudaStream_t side = h->split;
    if ((e = cudaStreamWaitEvent(side, h->split_ev[0], 0)) != cudaSuccess) return fail_cuda(h, e);
    char* reg = static_cast<char*>(d_work) + pp.bytes;
    std::vector<int> host(sp.ids);
    host.resize((size_t)count + 3 * (size_t)batch);
    for (int i = 0; i < batch; ++i) {
        host[count + i] = lda[i];
        host[count + batch + i] = wantU ? ldu[i] : 1;
        host[count + 2 * (size_t)batch + i] = wantV ? ldv[i] : 1;
    }
    int* dints = reinterpret_cast<int*>(reg);
    e = cudaMemcpyAsync(dints, host.data(), sizeof(int) * host.size(), cudaMemcpyHostToDevice, side);
    if (e == cudaSuccess) {
        BlockedArgs a = blocked_args(1, 1, count, wantU, wantV, r, true);
        a.Ap = dA; a.ldap = dints + count;
        a.Sp = dS;
        a.Up = dU; a.ldup = dints + count + batch;
        a.Vp = dV; a.ldvp = dints + count + 2 * batch;
        a.index = dints;
        a.info = d_info;
        a.sweeps = d_sweeps;
        e = ops.blocked_var(sp.nb, a, sp.var, reg + sp.ints, side, capture_stream(h, r.flags));
    }
    // join, also after a failure: the caller's stream owns the results
    cudaError_t ej = cudaEventRecord(h->split_ev[1], side);
    if (ej == cudaSuccess) ej = cudaStreamWaitEvent(s, h->split_ev[1], 0);
    if (e == cudaSuccess) e = ej;
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
    if (d_work && (reinterpret_cast<uintptr_t>(d_work) & 15) != 0) return fail_arg(h, 16);
    const TypeOps ops = ops_for(t);
    if (opts && (opts->flags & kFlagQR)) return BSVD_ERR_NOT_IMPLEMENTED;      // strided form only
    // MIXED runs per shape group (with PERSISTENT too): the mixed-precision
    // path of the strided form on each group, inputs and outputs through the
    // pointer arrays
    const bool mixed = opts && opts->prec == BSVD_PREC_MIXED;
    bsvd_opts om;
    if (mixed && opts->path == BSVD_PATH_PERSISTENT) {
        om = *opts;
        om.path = BSVD_PATH_AUTO;
        om.flags &= ~(kFlagSplit | kFlagSplitF32 | kFlagNoOnChip);
        opts = &om;
    }
    if (opts && opts->path == BSVD_PATH_PERSISTENT) {
        bsvd_status st = refresh_device(h);
        if (st != BSVD_OK) return st;
        if (split_large(ops, opts))
            return split_impl(h, t, ops, wantU, wantV, batch, m, n, dA, lda, dS, dU, ldu, dV, ldv, d_info,
                              d_sweeps, d_work, work_bytes, opts, static_cast<cudaStream_t>(stream));
        return persistent_impl(h, t, ops, wantU, wantV, batch, m, n, dA, lda, dS, dU, ldu, dV, ldv, d_info,
                               d_sweeps, d_work, work_bytes, opts, static_cast<cudaStream_t>(stream));
    }
    Groups groups;
    for (int i = 0; i < batch; ++i) groups[{m[i], n[i]}].push_back(i);
    // plan every group before touching the device, so a bad shape fails cleanly
    std::vector<Plan> plans;
    std::vector<Resolved> res;
    size_t need = 0;
    bsvd_status st = plan_batched(h, t, device_smem_or_default(h), ops, batch, groups, wantU, wantV,
                                  opts, plans, res, need);
    if (st == BSVD_ERR_INVALID) return fail_arg(h, 18);
    if (st != BSVD_OK) return st;
    if (!d_work || work_bytes < need) return BSVD_ERR_WORKSPACE;
    st = refresh_device(h);
    if (st != BSVD_OK) return st;
    cudaStream_t s = static_cast<cudaStream_t>(stream);

    std::vector<int> host((size_t)4 * batch);
    std::memcpy(host.data(), lda, sizeof(int) * batch);
    for (int i = 0; i < batch; ++i) {
        host[batch + i] = wantU ? ldu[i] : 1;
        host[2 * batch + i] = wantV ? ldv[i] : 1;
    }
    std::vector<size_t> ipos;
    size_t pos = 3 * (size_t)batch;
    for (auto& kv : groups) {
        ipos.push_back(pos);
        std::copy(kv.second.begin(), kv.second.end(), host.begin() + pos);
        pos += kv.second.size();
    }
    int* dws = static_cast<int*>(d_work);
    cudaError_t e = cudaMemcpyAsync(dws, host.data(), sizeof(int) * host.size(), cudaMemcpyHostToDevice, s);
    if (e != cudaSuccess) return fail_cuda(h, e);
    char* region = static_cast<char*>(d_work) + batched_ints(batch);
    size_t gi = 0;
    for (auto& kv : groups) {
        const int mm = kv.first.first, nn = kv.first.second;
        const int count = (int)kv.second.size();
        Plan& p = plans[gi];
        const Resolved& r = res[gi];
        const int* index = dws + ipos[gi];
        ++gi;
        if (std::min(mm, nn) == 0) {
            for (int id : kv.second) {
                e = cudaMemsetAsync(d_info + id, 0, sizeof(int), s);
                if (e == cudaSuccess && d_sweeps) e = cudaMemsetAsync(d_sweeps + id, 0, sizeof(int), s);
                if (e != cudaSuccess) return fail_cuda(h, e);
            }
            continue;
        }
        if (p.mixed) {
            const PtrIO io{reinterpret_cast<const void* const*>(dA), dws, dS, dU, dws + batch, dV, dws + 2 * batch,
                           index};
            bsvd_status sm = mixed_impl(t, h, wantU, wantV, count, mm, nn, nullptr, 1, 0, nullptr, 0, nullptr, 1, 0,
                                        nullptr, 1, 0, d_info, d_sweeps, region, p.bytes, r, s, &io);
            if (sm != BSVD_OK) return sm;
            region += align256(p.bytes);
            continue;
        }
        if (p.blocked) {
            BlockedArgs a = blocked_args(mm, nn, count, wantU, wantV, r, p.masks);
            a.Ap = dA; a.ldap = dws;
            a.Sp = dS;
            a.Up = dU; a.ldup = dws + batch;
            a.Vp = dV; a.ldvp = dws + 2 * batch;
            a.index = index;
            a.info = d_info;
            a.sweeps = d_sweeps;
            e = ops.blocked(p.nb, a, region, s, p.two_stage, p.host_sync, capture_stream(h, r.flags));
            region += align256(p.bytes);
        } else {
            FusedArgs& a = p.a;
            a.Ap = dA; a.ldap = dws;
            a.Sp = dS;
            a.Up = dU; a.ldup = dws + batch;
            a.Vp = dV; a.ldvp = dws + 2 * batch;
            a.index = index;
            a.info = d_info;
            a.sweeps = d_sweeps;
            e = ops.launch(p.nb, a, count, p.smem, s);
        }
        if (e != cudaSuccess) return fail_cuda(h, e);
    }
    return BSVD_OK;
}

}  // namespace

size_t bsvd::blocked_bytes(int nb, int M, int N, int count, bool two_stage, size_t elt) {
    return blk_bytes(nb, M, N, count, two_stage, elt);
}

bsvd_status bsvd::persistent_with_flags(bsvd_handle h, char t, bool wantU, bool wantV, int batch, const int* m,
                                        const int* n, const void* const* dA, const int* lda, void* const* dS,
                                        void* const* dU, const int* ldu, void* const* dV, const int* ldv,
                                        int* d_info, int* d_sweeps, int* d_done, const int* d_abort,
                                        void* d_work, size_t work_bytes, const bsvd_opts* opts, cudaStream_t s) {
    if (!h || batch < 1) return BSVD_ERR_INVALID;
    bsvd_status st = refresh_device(h);
    if (st != BSVD_OK) return st;
    return persistent_impl(h, t, ops_for(t), wantU, wantV, batch, m, n, dA, lda, dS, dU, ldu, dV, ldv, d_info,
                           d_sweeps, d_work, work_bytes, opts, s, d_done, d_abort);
}

namespace {

// Candidates of the autotuner: block width x {on-chip fused, multi-kernel}.
// The block width also sets the threads per matrix (64, 128 or 256 per CTA
// on chip; 128-thread update CTAs and 32-256-thread eigensolver CTAs on the
// multi-kernel path).
constexpr int kTuneCands = 8;
constexpr int kTuneBatch = 512;
void tune_cand(int c, int& path, int& nb) {
    static const int nbs[4] = {4, 8, 16, 32};
    nb = nbs[c / 2];
    path = (c % 2 == 0) ? BSVD_PATH_FUSED : BSVD_PATH_BLOCKED;
}

struct TuneLayout {
    size_t off[5];      // S, U, V, info, sweeps
    size_t cand_off;    // candidate workspace
    size_t bytes;
};

bsvd_status tune_layout(bsvd_handle h, char t, int tb, int m, int n, bool wantU, bool wantV,
                        const bsvd_opts* base, TuneLayout& L, bool feasible[kTuneCands]) {
    const TypeOps ops = ops_for(t);
    const int k = std::min(m, n);
    const size_t rsz = ops.single ? 4 : 8;
    const size_t sizes[5] = {(size_t)tb * k * rsz, wantU ? (size_t)tb * m * k * ops.elt : 0,
                             wantV ? (size_t)tb * n * k * ops.elt : 0, (size_t)tb * sizeof(int),
                             (size_t)tb * sizeof(int)};
    size_t pos = 0;
    for (int i = 0; i < 5; ++i) { L.off[i] = pos; pos += align256(sizes[i]); }
    L.cand_off = pos;
    size_t need = 0;
    const int max_smem = device_smem_or_default(h);
    for (int c = 0; c < kTuneCands; ++c) {
        bsvd_opts o;
        if (base) o = *base;
        else std::memset(&o, 0, sizeof o);
        tune_cand(c, o.path, o.nb);
        o.prec = BSVD_PREC_NATIVE;
        o.flags &= 1;
        feasible[c] = false;
        Resolved r;
        if (!resolve(&o, ops.single, k, r)) continue;
        if (r.nb > std::max(4, 2 * k)) continue;            // wider than the matrix: pointless
        Plan p;
        if (plan_group(max_smem, ops, m, n, tb, wantU, wantV, r, p) != BSVD_OK) continue;
        feasible[c] = true;
        if (p.blocked) need = std::max(need, p.bytes);
    }
    L.bytes = pos + align256(need);
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
    if (handle && handle->cap) cudaStreamDestroy(handle->cap);
    if (handle) {
        for (cudaStream_t s : handle->pipe)
            if (s) cudaStreamDestroy(s);
        if (handle->split) cudaStreamDestroy(handle->split);
        for (cudaEvent_t ev : handle->split_ev)
            if (ev) cudaEventDestroy(ev);
        for (cudaStream_t s : handle->pstream)
            if (s) cudaStreamDestroy(s);
        for (cudaEvent_t ev : handle->pevent)
            if (ev) cudaEventDestroy(ev);
        if (handle->pfork) cudaEventDestroy(handle->pfork);
    }
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
        case BSVD_ERR_CANCELLED: return "BSVD_ERR_CANCELLED: request cancelled";
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
    *bytes = 0;
    if (batch == 0) return BSVD_OK;
    const TypeOps ops = ops_for(dtype);
    const bool wantU = jobu == BSVD_JOB_SOME, wantV = jobv == BSVD_JOB_SOME;
    const int max_smem = device_smem_or_default(handle);
    if (uniform) {
        const int m = m_arr[0], n = n_arr[0];
        if (m < 0) return fail_arg(handle, 4);
        if (n < 0) return fail_arg(handle, 5);
        if (std::min(m, n) == 0) return BSVD_OK;
        Resolved r;
        if (!resolve(opts, ops.single, std::min(m, n), r)) return fail_arg(handle, 9);
        if (r.path == BSVD_PATH_PERSISTENT) r.path = BSVD_PATH_AUTO;   // as the strided call does
        apply_tuned(handle, dtype, m, n, wantU, wantV, opts, r);
        if (r.flags & kFlagQR) {
            if (r.prec == BSVD_PREC_MIXED) return BSVD_ERR_NOT_IMPLEMENTED;
            QrPlan qp;
            bsvd_status st = plan_qr(max_smem, ops, m, n, batch, wantU, wantV, r, qp);
            if (st == BSVD_OK) *bytes = qp.bytes;
            return st;
        }
        if (r.prec == BSVD_PREC_MIXED) {
            MixedPlan mp;
            bsvd_status st = plan_mixed(max_smem, dtype, m, n, batch, wantU, wantV, r, mp);
            if (st == BSVD_OK) *bytes = mp.bytes;
            return st;
        }
        Plan p;
        bsvd_status st = plan_group(max_smem, ops, m, n, batch, wantU, wantV, r, p);
        if (st != BSVD_OK) return st;
        *bytes = p.blocked ? p.bytes : 0;
        return BSVD_OK;
    }
    Groups groups;
    for (int i = 0; i < batch; ++i) {
        if (m_arr[i] < 0) return fail_arg(handle, 4);
        if (n_arr[i] < 0) return fail_arg(handle, 5);
        groups[{m_arr[i], n_arr[i]}].push_back(i);
    }
    if (opts && (opts->flags & kFlagQR)) return BSVD_ERR_NOT_IMPLEMENTED;      // strided form only
    bsvd_opts om;
    if (opts && opts->prec == BSVD_PREC_MIXED && opts->path == BSVD_PATH_PERSISTENT) {   // per shape group
        om = *opts;
        om.path = BSVD_PATH_AUTO;
        om.flags &= ~(kFlagSplit | kFlagSplitF32 | kFlagNoOnChip);
        opts = &om;
    }
    if (opts && opts->path == BSVD_PATH_PERSISTENT) {
        SplitPlan sp;
        const bool split = split_large(ops, opts);
        if (split) plan_split(ops, batch, m_arr, n_arr, opts, sp);
        PersistPlan pp;
        bsvd_status st = plan_persistent(handle, dtype, device_sms_or_default(handle), max_smem, ops, batch, m_arr,
                                         n_arr, wantU, wantV, opts, pp, split ? &sp.excl : nullptr);
        if (st == BSVD_OK) *bytes = pp.bytes + (split ? sp.bytes : 0);
        return st;
    }
    std::vector<Plan> plans;
    std::vector<Resolved> res;
    bsvd_status st = plan_batched(handle, dtype, max_smem, ops, batch, groups, wantU, wantV, opts, plans,
                                  res, *bytes);
    if (st == BSVD_ERR_INVALID) return fail_arg(handle, 9);
    return st;
}

bsvd_status bsvd_persistent_plan(bsvd_handle handle, char dtype, int batch, const int* m_arr, const int* n_arr,
                                 bsvd_job jobu, bsvd_job jobv, const bsvd_opts* opts, int* nb_out, int* where_out,
                                 int* launches) {
    if (!handle) return BSVD_ERR_INVALID;
    handle->last_arg = 0;
    if (dtype != 's' && dtype != 'd' && dtype != 'c' && dtype != 'z') return fail_arg(handle, 2);
    if (batch < 0) return fail_arg(handle, 3);
    if (batch > 0 && (!m_arr || !n_arr)) return fail_arg(handle, !m_arr ? 4 : 5);
    if (batch > 0 && (!nb_out || !where_out)) return fail_arg(handle, !nb_out ? 9 : 10);
    for (int i = 0; i < batch; ++i) {
        if (m_arr[i] < 0) return fail_arg(handle, 4);
        if (n_arr[i] < 0) return fail_arg(handle, 5);
    }
    const TypeOps ops = ops_for(dtype);
    const bool wantU = jobu == BSVD_JOB_SOME, wantV = jobv == BSVD_JOB_SOME;
    SplitPlan sp;
    const bool split = split_large(ops, opts);
    if (split) plan_split(ops, batch, m_arr, n_arr, opts, sp);
    PersistPlan pp;
    bsvd_status st = plan_persistent(handle, dtype, device_sms_or_default(handle), device_smem_or_default(handle),
                                     ops, batch, m_arr, n_arr, wantU, wantV, opts, pp, split ? &sp.excl : nullptr);
    if (st != BSVD_OK) return st;
    for (int i = 0; i < batch; ++i) {
        nb_out[i] = pp.nb_of[i];
        where_out[i] = pp.where_of[i];
        if (split && sp.excl[i]) {
            nb_out[i] = sp.nb;
            where_out[i] = 2;
        }
    }
    if (launches) *launches = (int)pp.segs.size();
    return BSVD_OK;
}

bsvd_status bsvd_autotune_workspace(bsvd_handle handle, char dtype, int batch, int m, int n,
                                    bsvd_job jobu, bsvd_job jobv, const bsvd_opts* base, size_t* bytes) {
    if (!handle) return BSVD_ERR_INVALID;
    handle->last_arg = 0;
    if (dtype != 's' && dtype != 'd' && dtype != 'c' && dtype != 'z') return fail_arg(handle, 2);
    if (batch < 1) return fail_arg(handle, 3);
    if (m < 1) return fail_arg(handle, 4);
    if (n < 1) return fail_arg(handle, 5);
    if (!bytes) return fail_arg(handle, 9);
    TuneLayout L;
    bool feas[kTuneCands];
    tune_layout(handle, dtype, std::min(batch, kTuneBatch), m, n, jobu == BSVD_JOB_SOME, jobv == BSVD_JOB_SOME,
                base, L, feas);
    *bytes = L.bytes;
    return BSVD_OK;
}

bsvd_status bsvd_autotune(bsvd_handle handle, char dtype, bsvd_job jobu, bsvd_job jobv, int batch, int m,
                          int n, const void* dA, int lda, long long strideA, void* d_work,
                          size_t work_bytes, const bsvd_opts* base, bsvd_opts* best, float* times_ms,
                          void* stream) {
    if (!handle) return BSVD_ERR_INVALID;
    handle->last_arg = 0;
    if (dtype != 's' && dtype != 'd' && dtype != 'c' && dtype != 'z') return fail_arg(handle, 2);
    if (jobu != BSVD_JOB_NONE && jobu != BSVD_JOB_SOME) return fail_arg(handle, 3);
    if (jobv != BSVD_JOB_NONE && jobv != BSVD_JOB_SOME) return fail_arg(handle, 4);
    if (batch < 1) return fail_arg(handle, 5);
    if (m < 1) return fail_arg(handle, 6);
    if (n < 1) return fail_arg(handle, 7);
    if (!dA) return fail_arg(handle, 8);
    if (lda < m) return fail_arg(handle, 9);
    if (batch > 1 && strideA < (long long)lda * n) return fail_arg(handle, 10);
    if (!best) return fail_arg(handle, 14);
    const bool wantU = jobu == BSVD_JOB_SOME, wantV = jobv == BSVD_JOB_SOME;
    const int tb = std::min(batch, kTuneBatch), k = std::min(m, n);
    bsvd_status st = refresh_device(handle);
    if (st != BSVD_OK) return st;
    TuneLayout L;
    bool feas[kTuneCands];
    tune_layout(handle, dtype, tb, m, n, wantU, wantV, base, L, feas);
    if (!d_work || work_bytes < L.bytes) return BSVD_ERR_WORKSPACE;
    char* w = static_cast<char*>(d_work);
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    cudaEvent_t e0, e1;
    if (cudaEventCreate(&e0) != cudaSuccess) return fail_cuda(handle, cudaGetLastError());
    if (cudaEventCreate(&e1) != cudaSuccess) { cudaEventDestroy(e0); return fail_cuda(handle, cudaGetLastError()); }
    std::vector<int> info(tb);
    int best_c = -1;
    float best_ms = 0.f;
    for (int c = 0; c < kTuneCands; ++c) {
        if (times_ms) times_ms[c] = -1.f;
        if (!feas[c]) continue;
        bsvd_opts o;
        if (base) o = *base;
        else std::memset(&o, 0, sizeof o);
        tune_cand(c, o.path, o.nb);
        o.prec = BSVD_PREC_NATIVE;
        o.flags &= 1;
        float ms = 0.f;
        bool ok = true;
        for (int rep = 0; rep < 2 && ok; ++rep) {      // the first run warms up, the second is timed
            cudaEventRecord(e0, s);
            st = strided_impl(dtype, handle, jobu, jobv, tb, m, n, dA, lda, strideA, w + L.off[0], k,
                              w + L.off[1], m, (long long)m * k, w + L.off[2], n, (long long)n * k,
                              reinterpret_cast<int*>(w + L.off[3]), reinterpret_cast<int*>(w + L.off[4]),
                              w + L.cand_off, L.bytes - L.cand_off, &o, stream);
            cudaEventRecord(e1, s);
            if (st != BSVD_OK || cudaEventSynchronize(e1) != cudaSuccess) { ok = false; break; }
            cudaEventElapsedTime(&ms, e0, e1);
        }
        if (!ok) { cudaGetLastError(); continue; }
        if (cudaMemcpy(info.data(), w + L.off[3], sizeof(int) * tb, cudaMemcpyDeviceToHost) != cudaSuccess) {
            cudaGetLastError();
            continue;
        }
        bool conv = true;                                    // every matrix must converge
        for (int v : info) conv = conv && v == 0;
        if (!conv) continue;
        if (times_ms) times_ms[c] = ms;
        if (best_c < 0 || ms < best_ms) { best_c = c; best_ms = ms; }
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    if (best_c < 0) return BSVD_ERR_NOT_IMPLEMENTED;
    bsvd_opts o;
    if (base) o = *base;
    else std::memset(&o, 0, sizeof o);
    tune_cand(best_c, o.path, o.nb);
    *best = o;
    handle->tuned[tune_key(dtype, m, n, wantU, wantV)] = bsvd_tuned{o.path, o.nb, best_ms};
    return BSVD_OK;
}


namespace {

// ---- autotuner for pointer-array batches of mixed shapes ---------------------
// Per bucket (type, M and N rounded up to powers of two, jobs) of the batch,
// persistent launches of a sample of the bucket's matrices are timed with
// each block width (4, 8, 16; the block width also fixes the threads per
// matrix: 64, 128 or 256 per CTA); on chip or in global slots follows from
// the fit at each width.  The winner is recorded in the handle and later
// persistent calls (and AUTO strided calls) of the bucket follow it.
constexpr int kTuneNbs[3] = {4, 8, 16};

struct BatchTuneBucket {
    bsvd_tune_key key;
    std::vector<int> ids;          // the sample (first matrices of the bucket)
};

struct BatchTuneLayout {
    std::vector<BatchTuneBucket> buckets;
    size_t bytes = 0;              // the largest sample's need
};

// Sample outputs (S, U, V per matrix, 256-byte aligned), pointer arrays,
// info and sweeps, then the persistent workspace of the candidate.
struct SampleLayout {
    std::vector<size_t> oS, oU, oV;
    size_t ptr_off = 0, info_off = 0, work_off = 0, bytes = 0;
};

size_t sample_layout(const TypeOps& ops, const std::vector<int>& ids, const int* m, const int* n, bool wantU,
                     bool wantV, SampleLayout& L) {
    const size_t rsz = ops.single ? 4 : 8;
    const size_t B = ids.size();
    size_t pos = 0;
    L.oS.resize(B); L.oU.resize(B); L.oV.resize(B);
    for (size_t i = 0; i < B; ++i) {
        const int mm = m[ids[i]], nn = n[ids[i]], k = std::min(mm, nn);
        L.oS[i] = pos; pos += align256((size_t)k * rsz);
        L.oU[i] = pos; if (wantU) pos += align256((size_t)mm * k * ops.elt);
        L.oV[i] = pos; if (wantV) pos += align256((size_t)nn * k * ops.elt);
    }
    L.ptr_off = pos; pos += 4 * align256(B * sizeof(void*));
    L.info_off = pos; pos += align256(2 * B * sizeof(int));
    L.work_off = pos;
    return pos;
}

bsvd_opts tune_opts(const bsvd_opts* base, int nb) {
    bsvd_opts o;
    if (base) o = *base;
    else std::memset(&o, 0, sizeof o);
    o.path = BSVD_PATH_PERSISTENT;
    o.nb = nb;
    o.prec = BSVD_PREC_NATIVE;
    o.flags &= (1 | 128 | 256 | 512);   // numerics and on-chip choice; no split, QR or host checks
    return o;
}

void batch_tune_layout(bsvd_handle h, char t, int batch, const int* m, const int* n, bool wantU, bool wantV,
                       const bsvd_opts* base, int sample, BatchTuneLayout& BL) {
    const TypeOps ops = ops_for(t);
    std::map<bsvd_tune_key, std::vector<int>> by;
    for (int i = 0; i < batch; ++i)
        if (std::min(m[i], n[i]) > 0) by[tune_key(t, m[i], n[i], wantU, wantV)].push_back(i);
    BL = BatchTuneLayout();
    for (auto& kv : by) {
        BatchTuneBucket b;
        b.key = kv.first;
        // the sample: at most `sample` matrices, and for large shapes no more
        // than about 64 matrices of 64 x 64 worth of work (M N^2), at least 2
        const int M = std::get<1>(kv.first), N = std::get<2>(kv.first);
        const double per = (double)M * N * N, budget = 64.0 * 64 * 64 * 64;
        const size_t cap = (size_t)std::max(2.0, std::min((double)sample, budget / per));
        b.ids.assign(kv.second.begin(), kv.second.begin() + std::min(kv.second.size(), cap));
        SampleLayout L;
        const size_t fixed = sample_layout(ops, b.ids, m, n, wantU, wantV, L);
        std::vector<int> sm, sn;
        for (int id : b.ids) { sm.push_back(m[id]); sn.push_back(n[id]); }
        for (int nb : kTuneNbs) {
            const bsvd_opts o = tune_opts(base, nb);
            PersistPlan pp;
            if (plan_persistent(h, t, device_sms_or_default(h), device_smem_or_default(h), ops, (int)b.ids.size(),
                                sm.data(), sn.data(), wantU, wantV, &o, pp) == BSVD_OK)
                BL.bytes = std::max(BL.bytes, fixed + pp.bytes);
        }
        BL.buckets.push_back(std::move(b));
    }
}

}  // namespace

bsvd_status bsvd_autotune_batched_workspace(bsvd_handle handle, char dtype, int batch, const int* m, const int* n,
                                            bsvd_job jobu, bsvd_job jobv, const bsvd_opts* base, int sample,
                                            size_t* bytes) {
    if (!handle) return BSVD_ERR_INVALID;
    handle->last_arg = 0;
    if (dtype != 's' && dtype != 'd' && dtype != 'c' && dtype != 'z') return fail_arg(handle, 2);
    if (batch < 0) return fail_arg(handle, 3);
    if (batch > 0 && (!m || !n)) return fail_arg(handle, !m ? 4 : 5);
    if (sample < 1) return fail_arg(handle, 9);
    if (!bytes) return fail_arg(handle, 10);
    for (int i = 0; i < batch; ++i)
        if (m[i] < 0 || n[i] < 0) return fail_arg(handle, m[i] < 0 ? 4 : 5);
    BatchTuneLayout BL;
    batch_tune_layout(handle, dtype, batch, m, n, jobu == BSVD_JOB_SOME, jobv == BSVD_JOB_SOME, base, sample, BL);
    *bytes = BL.bytes;
    return BSVD_OK;
}

bsvd_status bsvd_autotune_batched(bsvd_handle handle, char dtype, bsvd_job jobu, bsvd_job jobv, int batch,
                                  const int* m, const int* n, const void* const* dA, const int* lda, void* d_work,
                                  size_t work_bytes, const bsvd_opts* base, int sample, int max_out,
                                  int* bucket_mn, int* nb_out, float* times_ms, int* buckets, void* stream) {
    if (!handle) return BSVD_ERR_INVALID;
    handle->last_arg = 0;
    if (dtype != 's' && dtype != 'd' && dtype != 'c' && dtype != 'z') return fail_arg(handle, 2);
    if (jobu != BSVD_JOB_NONE && jobu != BSVD_JOB_SOME) return fail_arg(handle, 3);
    if (jobv != BSVD_JOB_NONE && jobv != BSVD_JOB_SOME) return fail_arg(handle, 4);
    if (batch < 0) return fail_arg(handle, 5);
    if (batch > 0 && (!m || !n || !dA || !lda)) return fail_arg(handle, !m ? 6 : !n ? 7 : !dA ? 8 : 9);
    if (sample < 1) return fail_arg(handle, 13);
    if (max_out < 0) return fail_arg(handle, 14);
    for (int i = 0; i < batch; ++i) {
        if (m[i] < 0) return fail_arg(handle, 6);
        if (n[i] < 0) return fail_arg(handle, 7);
        if (lda[i] < std::max(1, m[i])) return fail_arg(handle, 9);
    }
    const bool wantU = jobu == BSVD_JOB_SOME, wantV = jobv == BSVD_JOB_SOME;
    bsvd_status st = refresh_device(handle);
    if (st != BSVD_OK) return st;
    BatchTuneLayout BL;
    batch_tune_layout(handle, dtype, batch, m, n, wantU, wantV, base, sample, BL);
    if (buckets) *buckets = (int)BL.buckets.size();
    if (batch == 0 || BL.buckets.empty()) return BSVD_OK;
    if (!d_work || work_bytes < BL.bytes) return BSVD_ERR_WORKSPACE;
    const TypeOps ops = ops_for(dtype);
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    // the caller's matrix pointers, to pick each sample's
    std::vector<const void*> hA(batch);
    cudaError_t e = cudaMemcpyAsync(hA.data(), dA, batch * sizeof(void*), cudaMemcpyDeviceToHost, s);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);
    if (e != cudaSuccess) return fail_cuda(handle, e);
    cudaEvent_t e0, e1;
    if (cudaEventCreate(&e0) != cudaSuccess) return fail_cuda(handle, cudaGetLastError());
    if (cudaEventCreate(&e1) != cudaSuccess) { cudaEventDestroy(e0); return fail_cuda(handle, cudaGetLastError()); }
    char* w = static_cast<char*>(d_work);
    for (size_t bi = 0; bi < BL.buckets.size(); ++bi) {
        const BatchTuneBucket& b = BL.buckets[bi];
        const bool out = (int)bi < max_out;
        if (out && bucket_mn) {
            bucket_mn[2 * bi] = std::get<1>(b.key);
            bucket_mn[2 * bi + 1] = std::get<2>(b.key);
        }
        if (out && nb_out) nb_out[bi] = 0;
        const int B = (int)b.ids.size();
        SampleLayout L;
        sample_layout(ops, b.ids, m, n, wantU, wantV, L);
        std::vector<const void*> pA(B);
        std::vector<void*> pS(B), pU(B), pV(B);
        std::vector<int> sm(B), sn(B), ints(3 * (size_t)B);   // lda, ldu, ldv (host; copied by the call)
        for (int i = 0; i < B; ++i) {
            const int id = b.ids[i];
            sm[i] = m[id]; sn[i] = n[id];
            pA[i] = hA[id];
            pS[i] = w + L.oS[i]; pU[i] = w + L.oU[i]; pV[i] = w + L.oV[i];
            ints[i] = lda[id]; ints[B + i] = std::max(1, m[id]); ints[2 * B + i] = std::max(1, n[id]);
        }
        const size_t pa = align256((size_t)B * sizeof(void*));
        void** dpA = reinterpret_cast<void**>(w + L.ptr_off);
        void** dpS = reinterpret_cast<void**>(w + L.ptr_off + pa);
        void** dpU = reinterpret_cast<void**>(w + L.ptr_off + 2 * pa);
        void** dpV = reinterpret_cast<void**>(w + L.ptr_off + 3 * pa);
        int* dinfo = reinterpret_cast<int*>(w + L.info_off);
        e = cudaMemcpyAsync(dpA, pA.data(), B * sizeof(void*), cudaMemcpyHostToDevice, s);
        if (e == cudaSuccess) e = cudaMemcpyAsync(dpS, pS.data(), B * sizeof(void*), cudaMemcpyHostToDevice, s);
        if (e == cudaSuccess) e = cudaMemcpyAsync(dpU, pU.data(), B * sizeof(void*), cudaMemcpyHostToDevice, s);
        if (e == cudaSuccess) e = cudaMemcpyAsync(dpV, pV.data(), B * sizeof(void*), cudaMemcpyHostToDevice, s);
        if (e == cudaSuccess) e = cudaStreamSynchronize(s);   // the host vectors go out of scope below
        if (e != cudaSuccess) break;
        int best_nb = 0;
        float best_ms = 0.f;
        const int kb = std::get<2>(b.key);                    // N rounded up to a power of two
        for (int c = 0; c < 3; ++c) {
            const int nb = kTuneNbs[c];
            if (out && times_ms) times_ms[3 * bi + c] = -1.f;
            // candidates near the shape: nb = 4 only up to 32 columns, nb = 16
            // from 16 columns on (others pad or serialise far too much)
            if ((nb == 4 && kb > 32) || (nb == 16 && kb < 16)) continue;
            const bsvd_opts o = tune_opts(base, nb);
            float ms = 0.f;
            bool ok = true;
            for (int rep = 0; rep < 2 && ok; ++rep) {       // the first run warms up, the second is timed
                cudaEventRecord(e0, s);
                st = persistent_impl(handle, dtype, ops, wantU, wantV, B, sm.data(), sn.data(),
                                     reinterpret_cast<const void* const*>(dpA), ints.data(), dpS, dpU,
                                     ints.data() + B, dpV, ints.data() + 2 * B, dinfo, dinfo + B,
                                     w + L.work_off, work_bytes - L.work_off, &o, s);
                cudaEventRecord(e1, s);
                if (st != BSVD_OK || cudaEventSynchronize(e1) != cudaSuccess) { ok = false; break; }
                cudaEventElapsedTime(&ms, e0, e1);
            }
            if (!ok) { cudaGetLastError(); continue; }
            std::vector<int> info(B);
            if (cudaMemcpy(info.data(), dinfo, sizeof(int) * B, cudaMemcpyDeviceToHost) != cudaSuccess) {
                cudaGetLastError();
                continue;
            }
            bool conv = true;                                    // every matrix must converge
            for (int v : info) conv = conv && v == 0;
            if (!conv) continue;
            if (out && times_ms) times_ms[3 * bi + c] = ms;
            if (best_nb == 0 || ms < best_ms) { best_nb = nb; best_ms = ms; }
        }
        if (best_nb) {
            handle->tuned[b.key] = bsvd_tuned{BSVD_PATH_AUTO, best_nb, best_ms};
            if (out && nb_out) nb_out[bi] = best_nb;
        }
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    if (e != cudaSuccess) return fail_cuda(handle, e);
    return BSVD_OK;
}

namespace {

// ---- strided batch with host buffers: a chunked copy / compute pipeline -------
struct HostPlan {
    int chunk = 0, nchunks = 0;
    size_t off[7];        // A, S, U, V, info, sweeps, solver workspace (one buffer set)
    size_t set_bytes = 0, bytes = 0;
};

bsvd_status plan_host(bsvd_handle h, char t, int batch, int m, int n, bool wantU, bool wantV, const bsvd_opts* opts,
                      HostPlan& hp) {
    const TypeOps ops = ops_for(t);
    const size_t e = ops.elt, re_ = ops.single ? 4 : 8;
    const int k = std::min(m, n);
    // 4 chunks of at least 4 waves of CTAs each; alternate chunks run on two
    // compute streams so one chunk's tail overlaps the next chunk's start
    const int minc = 4 * device_sms_or_default(h);
    hp.chunk = std::max(1, std::min(batch, std::max(minc, (batch + 3) / 4)));
    hp.nchunks = (batch + hp.chunk - 1) / hp.chunk;
    int mm[1] = {m}, nn[1] = {n};
    size_t ws = 0;
    bsvd_status st = bsvd_gesvj_workspace(h, t, hp.chunk, mm, nn, 1, wantU ? BSVD_JOB_SOME : BSVD_JOB_NONE,
                                          wantV ? BSVD_JOB_SOME : BSVD_JOB_NONE, opts, &ws);
    if (st != BSVD_OK) return st;
    const size_t c = (size_t)hp.chunk;
    const size_t sizes[7] = {c * m * n * e, c * k * re_, wantU ? c * m * k * e : 0, wantV ? c * n * k * e : 0,
                             c * sizeof(int), c * sizeof(int), ws};
    size_t pos = 0;
    for (int i = 0; i < 7; ++i) { hp.off[i] = pos; pos += align256(std::max<size_t>(sizes[i], 1)); }
    hp.set_bytes = pos;
    hp.bytes = (hp.nchunks > 1 ? 2 : 1) * pos;
    return BSVD_OK;
}

cudaError_t pipe_streams(bsvd_handle h) {
    if (h->pipe[0] && h->pipe_device == h->device) return cudaSuccess;
    for (cudaStream_t& s : h->pipe) {
        if (s) cudaStreamDestroy(s);
        s = nullptr;
    }
    for (cudaStream_t& s : h->pipe) {
        const cudaError_t e = cudaStreamCreateWithFlags(&s, cudaStreamNonBlocking);
        if (e != cudaSuccess) return e;
    }
    h->pipe_device = h->device;
    return cudaSuccess;
}

// Copy of `count` matrices rows x cols (column pitch ld, matrix stride sd,
// element e bytes) between host and device layouts.
cudaError_t copy_mats(void* dst, size_t dld, long long dsd, const void* src, size_t sld, long long ssd, int rows,
                      int cols, int count, size_t e, cudaMemcpyKind kind, cudaStream_t s) {
    if (rows == 0 || cols == 0 || count == 0) return cudaSuccess;
    if (dsd == (long long)dld * cols && ssd == (long long)sld * cols)   // one pitched copy of count * cols columns
        return cudaMemcpy2DAsync(dst, dld * e, src, sld * e, rows * e, (size_t)cols * count, kind, s);
    for (int i = 0; i < count; ++i) {
        const cudaError_t err = cudaMemcpy2DAsync(static_cast<char*>(dst) + (size_t)i * dsd * e, dld * e,
                                                  static_cast<const char*>(src) + (size_t)i * ssd * e, sld * e,
                                                  rows * e, cols, kind, s);
        if (err != cudaSuccess) return err;
    }
    return cudaSuccess;
}

bsvd_status host_impl(char t, bsvd_handle h, bsvd_job jobu, bsvd_job jobv, int batch, int m, int n, const void* hA,
                      int lda, long long sA, void* hS, long long sS, void* hU, int ldu, long long sU, void* hV,
                      int ldv, long long sV, int* h_info, int* h_sweeps, void* d_work, size_t work_bytes,
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
    if (batch > 0 && m > 0 && n > 0 && !hA) return fail_arg(h, 7);
    if (lda < std::max(1, m)) return fail_arg(h, 8);
    if (batch > 1 && sA < (long long)lda * n) return fail_arg(h, 9);
    if (batch > 0 && k > 0 && !hS) return fail_arg(h, 10);
    if (batch > 1 && sS < k) return fail_arg(h, 11);
    if (wantU && batch > 0 && k > 0 && !hU) return fail_arg(h, 12);
    if (wantU && ldu < std::max(1, m)) return fail_arg(h, 13);
    if (wantU && batch > 1 && sU < (long long)ldu * k) return fail_arg(h, 14);
    if (wantV && batch > 0 && k > 0 && !hV) return fail_arg(h, 15);
    if (wantV && ldv < std::max(1, n)) return fail_arg(h, 16);
    if (wantV && batch > 1 && sV < (long long)ldv * k) return fail_arg(h, 17);
    if (batch > 0 && !h_info) return fail_arg(h, 18);
    if (d_work && (reinterpret_cast<uintptr_t>(d_work) & 255) != 0) return fail_arg(h, 20);
    Resolved r;
    if (!resolve(opts, ops_for(t).single, k, r)) return fail_arg(h, 22);
    if (batch == 0 || k == 0) return BSVD_OK;
    if (batch == 1) {   // strides are not used: make them the packed ones
        sA = (long long)lda * n; sS = k; sU = (long long)ldu * k; sV = (long long)ldv * k;
    }
    bsvd_status st = refresh_device(h);
    if (st != BSVD_OK) return st;
    HostPlan hp;
    st = plan_host(h, t, batch, m, n, wantU, wantV, opts, hp);
    if (st != BSVD_OK) return st;
    if (!d_work || work_bytes < hp.bytes) return BSVD_ERR_WORKSPACE;
    cudaError_t e = pipe_streams(h);
    if (e != cudaSuccess) return fail_cuda(h, e);
    const TypeOps ops = ops_for(t);
    const size_t el = ops.elt, rel = ops.single ? 4 : 8;
    cudaStream_t s0 = static_cast<cudaStream_t>(stream), h2d = h->pipe[0], d2h = h->pipe[1], s1 = h->pipe[2];
    const int C = hp.nchunks;
    std::vector<cudaEvent_t> ev_h2d(C), ev_comp(C), ev_d2h(C);
    cudaEvent_t start = nullptr;
    auto cleanup = [&]() {
        for (int c = 0; c < C; ++c) {
            if (ev_h2d[c]) cudaEventDestroy(ev_h2d[c]);
            if (ev_comp[c]) cudaEventDestroy(ev_comp[c]);
            if (ev_d2h[c]) cudaEventDestroy(ev_d2h[c]);
        }
        if (start) cudaEventDestroy(start);
    };
    auto ck = [&](cudaError_t err) { if (err != cudaSuccess && e == cudaSuccess) e = err; return err == cudaSuccess; };
    ck(cudaEventCreateWithFlags(&start, cudaEventDisableTiming));
    for (int c = 0; c < C && e == cudaSuccess; ++c) {
        ck(cudaEventCreateWithFlags(&ev_h2d[c], cudaEventDisableTiming));
        ck(cudaEventCreateWithFlags(&ev_comp[c], cudaEventDisableTiming));
        ck(cudaEventCreateWithFlags(&ev_d2h[c], cudaEventDisableTiming));
    }
    // the pipeline's streams start after what the caller queued on `stream`
    if (e == cudaSuccess && ck(cudaEventRecord(start, s0)))
        for (cudaStream_t x : {h2d, d2h, s1}) ck(cudaStreamWaitEvent(x, start, 0));
    char* w = static_cast<char*>(d_work);
    auto set = [&](int c) { return w + (size_t)(c & 1) * hp.set_bytes; };
    auto rows_of = [&](int c) { return std::min(hp.chunk, batch - c * hp.chunk); };
    auto h2d_chunk = [&](int c) {
        if (c >= 2) ck(cudaStreamWaitEvent(h2d, ev_comp[c - 2], 0));          // the buffer's A is free
        const long long i0 = (long long)c * hp.chunk;
        ck(copy_mats(set(c) + hp.off[0], m, (long long)m * n, static_cast<const char*>(hA) + i0 * sA * el, lda, sA,
                     m, n, rows_of(c), el, cudaMemcpyHostToDevice, h2d));
        ck(cudaEventRecord(ev_h2d[c], h2d));
    };
    auto compute_chunk = [&](int c) -> bsvd_status {
        cudaStream_t cs = (c & 1) ? s1 : s0;
        ck(cudaStreamWaitEvent(cs, ev_h2d[c], 0));
        if (c >= 2) ck(cudaStreamWaitEvent(cs, ev_d2h[c - 2], 0));             // the buffer's outputs are read out
        if (e != cudaSuccess) return BSVD_ERR_CUDA;
        char* b = set(c);
        const bsvd_status rs = strided_impl(t, h, jobu, jobv, rows_of(c), m, n, b + hp.off[0], std::max(1, m),
                                            (long long)m * n, b + hp.off[1], k, b + hp.off[2], std::max(1, m),
                                            (long long)m * k, b + hp.off[3], std::max(1, n), (long long)n * k,
                                            reinterpret_cast<int*>(b + hp.off[4]), reinterpret_cast<int*>(b + hp.off[5]),
                                            b + hp.off[6], hp.set_bytes - hp.off[6], opts, cs);
        if (rs != BSVD_OK) return rs;
        ck(cudaEventRecord(ev_comp[c], cs));
        return BSVD_OK;
    };
    auto d2h_chunk = [&](int c) {
        ck(cudaStreamWaitEvent(d2h, ev_comp[c], 0));
        const long long i0 = (long long)c * hp.chunk;
        const int cnt = rows_of(c);
        char* b = set(c);
        ck(copy_mats(static_cast<char*>(hS) + i0 * sS * rel, sS, sS, b + hp.off[1], k, k, k, 1, cnt, rel,
                     cudaMemcpyDeviceToHost, d2h));
        if (wantU) ck(copy_mats(static_cast<char*>(hU) + i0 * sU * el, ldu, sU, b + hp.off[2], m, (long long)m * k,
                                m, k, cnt, el, cudaMemcpyDeviceToHost, d2h));
        if (wantV) ck(copy_mats(static_cast<char*>(hV) + i0 * sV * el, ldv, sV, b + hp.off[3], n, (long long)n * k,
                                n, k, cnt, el, cudaMemcpyDeviceToHost, d2h));
        ck(cudaMemcpyAsync(h_info + i0, b + hp.off[4], cnt * sizeof(int), cudaMemcpyDeviceToHost, d2h));
        if (h_sweeps) ck(cudaMemcpyAsync(h_sweeps + i0, b + hp.off[5], cnt * sizeof(int), cudaMemcpyDeviceToHost, d2h));
        ck(cudaEventRecord(ev_d2h[c], d2h));
    };
    bsvd_status rs = BSVD_OK;
    for (int c = 0; c < std::min(C, 2) && e == cudaSuccess && rs == BSVD_OK; ++c) {
        h2d_chunk(c);
        rs = compute_chunk(c);
    }
    for (int c = 0; c < C && e == cudaSuccess && rs == BSVD_OK; ++c) {
        d2h_chunk(c);
        if (c + 2 < C) {
            h2d_chunk(c + 2);
            rs = compute_chunk(c + 2);
        }
    }
    // `stream` reaches the end of the call after every copy out
    if (e == cudaSuccess && rs == BSVD_OK)
        for (int c = std::max(0, C - 2); c < C; ++c) ck(cudaStreamWaitEvent(s0, ev_d2h[c], 0));
    cleanup();
    if (rs != BSVD_OK) return rs;
    return e == cudaSuccess ? BSVD_OK : fail_cuda(h, e);
}

}  // namespace

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

bsvd_status bsvd_gesvj_host_workspace(bsvd_handle handle, char dtype, int batch, int m, int n, bsvd_job jobu,
                                      bsvd_job jobv, const bsvd_opts* opts, size_t* bytes) {
    if (!handle) return BSVD_ERR_INVALID;
    handle->last_arg = 0;
    if (dtype != 's' && dtype != 'd' && dtype != 'c' && dtype != 'z') return fail_arg(handle, 2);
    if (batch < 0) return fail_arg(handle, 3);
    if (m < 0) return fail_arg(handle, 4);
    if (n < 0) return fail_arg(handle, 5);
    if (!bytes) return fail_arg(handle, 9);
    *bytes = 0;
    if (batch == 0 || std::min(m, n) == 0) return BSVD_OK;
    HostPlan hp;
    const bsvd_status st = plan_host(handle, dtype, batch, m, n, jobu == BSVD_JOB_SOME, jobv == BSVD_JOB_SOME,
                                     opts, hp);
    if (st == BSVD_OK) *bytes = hp.bytes;
    return st;
}

#define BSVD_HOST_IMPL(TAG, T, R)                                                              \
    bsvd_status bsvd_##TAG##gesvj_strided_host(BSVD_STRIDED_HOST_ARGS(T, R)) {                  \
        return host_impl(#TAG[0], handle, jobu, jobv, batch, m, n, hA, lda, strideA, hS,        \
                         strideS, hU, ldu, strideU, hV, ldv, strideV, h_info, h_sweeps,         \
                         d_work, work_bytes, opts, stream);                                     \
    }
BSVD_HOST_IMPL(s, float, float)
BSVD_HOST_IMPL(d, double, double)
BSVD_HOST_IMPL(c, void, float)
BSVD_HOST_IMPL(z, void, double)

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
