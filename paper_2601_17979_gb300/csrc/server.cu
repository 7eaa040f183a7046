// server.cu -- the serving loop of include/bsvd.h: a request queue, admission
// by the caller's device-memory arena, continuous batching over several
// streams, and per-request completion from flags the persistent kernel
// raises in host-mapped memory.
//
// Threads: callers submit / wait / collect / release under the server mutex;
// one worker thread owns the library handle and every launch.  The worker
// loops: retire what finished (flags of running persistent batches, events
// of batches that ended), admit what fits (oldest request first, its key's
// queue taken up to max_batch), launch, then sleep until a submit or a
// release wakes it or, with batches running, for a short poll interval.
#include <cuda_runtime.h>

#include <algorithm>
#include <atomic>
#include <chrono>
#include <condition_variable>
#include <cstdint>
#include <cstring>
#include <deque>
#include <map>
#include <memory>
#include <mutex>
#include <new>
#include <thread>
#include <tuple>
#include <vector>

#include "bsvd.h"
#include "internal.h"

namespace {

using Clock = std::chrono::steady_clock;

double now_s() { return std::chrono::duration<double>(Clock::now().time_since_epoch()).count(); }

size_t elt_size(char t) { return t == 's' ? 4 : (t == 'd' || t == 'c') ? 8 : 16; }
size_t real_size(char t) { return (t == 's' || t == 'c') ? 4 : 8; }
size_t align256(size_t x) { return (x + 255) & ~size_t(255); }
int auto_nb(int k) { return k >= 48 ? 16 : (k >= 12 ? 8 : 4); }

// First-fit allocator over [0, size) with coalescing of free neighbours.
class Arena {
public:
    explicit Arena(size_t size) : size_(size) { free_[0] = size; }
    bool alloc(size_t bytes, size_t& off) {
        bytes = align256(std::max<size_t>(bytes, 1));
        for (auto it = free_.begin(); it != free_.end(); ++it)
            if (it->second >= bytes) {
                off = it->first;
                const size_t rest = it->second - bytes;
                free_.erase(it);
                if (rest) free_[off + bytes] = rest;
                used_ += bytes;
                peak_ = std::max(peak_, used_);
                return true;
            }
        return false;
    }
    void release(size_t off, size_t bytes) {
        bytes = align256(std::max<size_t>(bytes, 1));
        used_ -= bytes;
        auto it = free_.emplace(off, bytes).first;
        auto nx = std::next(it);
        if (nx != free_.end() && it->first + it->second == nx->first) {
            it->second += nx->second;
            free_.erase(nx);
        }
        if (it != free_.begin()) {
            auto pv = std::prev(it);
            if (pv->first + pv->second == it->first) {
                pv->second += it->second;
                free_.erase(it);
            }
        }
    }
    size_t size() const { return size_; }
    size_t used() const { return used_; }
    size_t peak() const { return peak_; }

private:
    size_t size_, used_ = 0, peak_ = 0;
    std::map<size_t, size_t> free_;   // offset -> length
};

enum State { kQueued, kRunning, kDone, kFailed };

struct OutBlock {
    size_t off = 0, bytes = 0;
    int refs = 0;                  // unreleased requests + 1 while the batch runs
};

struct Request {
    long long id = 0;
    char dtype = 'd';
    int m = 0, n = 0, k = 0, lda = 0;
    const void* A = nullptr;       // device-accessible address
    bool wantU = false, wantV = false;
    double t_submit = 0, t_done = 0;
    int info = 0, sweeps = 0, status = 0;
    State state = kQueued;
    OutBlock* out = nullptr;
    char* S = nullptr;
    char* U = nullptr;
    char* V = nullptr;
};

// Batch key: type, jobs, block width; for the multi-kernel path also the shape.
using Key = std::tuple<char, int, int, int, int, int>;   // dtype, jobs, nb, big, m, n

// What a launch reads: the requests, their stream slot and the workspace.
struct Job {
    std::vector<Request*> reqs;
    bool persistent = true;
    int slot = -1;
    size_t ws_off = 0, ws_bytes = 0;
};

struct Batch : Job {
    std::vector<int> pending;      // indices of requests not yet retired
    OutBlock* out = nullptr;
    std::thread launcher;          // multi-kernel batches are launched off the worker thread
};

}  // namespace

struct bsvd_server_s {
    bsvd_handle h = nullptr;
    int device = 0;
    char* arena_base = nullptr;
    Arena* arena = nullptr;
    int max_inflight = 32, max_batch = 4096, big_k = 256, max_big_batch = 8, fp64_prec = 0, big_flags = 0;
    int big_k_fp64 = 256;
    // per slot two streams: high priority for persistent batches (small
    // requests), low priority for multi-kernel batches (large ones), so the
    // block scheduler starts a small request's CTAs before a large batch's
    std::vector<cudaStream_t> streams, streams_lo;
    std::vector<cudaEvent_t> events;
    std::vector<int*> hflags;      // per slot, host-mapped: info, sweeps, done (max_batch each), abort
    std::vector<int*> dflags;      // the same memory's device addresses
    std::vector<bool> slot_busy;
    std::vector<bool> slot_abort;  // the slot's batch was told to stop
    std::vector<bool> slot_big;    // the slot runs a multi-kernel batch
    std::vector<bsvd_handle> slot_h;                      // one library handle per stream
    std::unique_ptr<std::atomic<int>[]> launch_state;     // per slot: 0 launching, 1 launched, < 0 failed
    std::vector<int> launch_cuda;                         // per slot: cudaError_t of a failed launch
    int big_cap = 12;              // slots multi-kernel batches may hold at once
    cudaStream_t fetch_stream = nullptr;

    std::mutex mu;
    std::condition_variable cv_work, cv_done;
    std::map<Key, std::deque<Request*>> queues;
    std::map<long long, Request*> reqs;
    std::deque<long long> completions;
    std::vector<Batch> running;
    long long next_id = 1, submitted = 0, completed = 0, failed = 0, cancelled = 0, launched = 0;
    long long queued = 0, in_flight = 0;
    bool stop = false, paused = false;
    long long wake_gen = 0;        // bumped (under mu) by every submit, release, pause and cancel
    std::thread worker;
};

namespace {

Key key_of(const bsvd_server_s* s, const Request* r) {
    const bool big = r->k > ((r->dtype == 'd' || r->dtype == 'z') ? s->big_k_fp64 : s->big_k);
    return Key(r->dtype, (r->wantU ? 1 : 0) | (r->wantV ? 2 : 0), big ? 16 : auto_nb(r->k), big ? 1 : 0,
               big ? r->m : 0, big ? r->n : 0);
}

size_t out_bytes(const Request* r) {
    const size_t e = elt_size(r->dtype);
    size_t b = align256((size_t)r->k * real_size(r->dtype));
    if (r->wantU) b += align256((size_t)r->m * r->k * e);
    if (r->wantV) b += align256((size_t)r->n * r->k * e);
    return b;
}

bsvd_opts batch_opts(const bsvd_server_s* s, const Request* r0, bool persistent) {
    bsvd_opts o;
    std::memset(&o, 0, sizeof o);
    o.nb = persistent ? auto_nb(r0->k) : 16;
    o.path = persistent ? BSVD_PATH_PERSISTENT : BSVD_PATH_AUTO;
    // persistent batches keep W and V in global slots (flags bit 9): their
    // CTAs then take little shared memory, so the CTAs of many batches share
    // the SMs and a newly admitted batch starts while older ones run;
    // multi-kernel batches stop issuing sweeps once converged (bit 4, for
    // the fallback without the device-side loop)
    // multi-kernel batches replay a one-sweep graph from their launcher
    // thread and stop once converged (bits 11 and 4): measured on the
    // request stream, tens of batches each running a graph with a device-side
    // conditional loop on its own stream held back the other streams' work
    // (at 50 requests/s the median small request took 144 ms against 0.7 ms)
    o.flags = persistent ? 512 : 16 | 2048 | s->big_flags;
    if (!persistent && (r0->dtype == 'd' || r0->dtype == 'z')) o.prec = s->fp64_prec;
    return o;
}

// Workspace of a batch: four pointer arrays, then the solver's workspace
// (0 if the solver cannot plan the batch).
size_t ws_bytes(const bsvd_server_s* s, bsvd_handle h, const std::vector<Request*>& rs, bool persistent) {
    std::vector<int> mm, nn;
    for (const Request* r : rs) {
        mm.push_back(r->m);
        nn.push_back(r->n);
    }
    const Request* r0 = rs.front();
    const bsvd_opts o = batch_opts(s, r0, persistent);
    size_t w = 0;
    if (bsvd_gesvj_workspace(h, r0->dtype, (int)rs.size(), mm.data(), nn.data(), 0,
                             r0->wantU ? BSVD_JOB_SOME : BSVD_JOB_NONE, r0->wantV ? BSVD_JOB_SOME : BSVD_JOB_NONE,
                             &o, &w) != BSVD_OK)
        return 0;
    return 4 * align256(rs.size() * sizeof(void*)) + align256(std::max<size_t>(w, 16));
}

size_t flag_ints(const bsvd_server_s* s) { return 3 * (size_t)s->max_batch + 1; }

void complete(bsvd_server_s* s, Request* r, int status) {
    r->t_done = now_s();
    r->status = status;
    r->state = status == BSVD_OK ? kDone : kFailed;
    if (status == BSVD_OK) s->completed++;
    else if (status == BSVD_ERR_CANCELLED) s->cancelled++;
    else s->failed++;
    s->completions.push_back(r->id);
}

void drop_out(bsvd_server_s* s, OutBlock*& ob) {
    if (ob && --ob->refs == 0) {
        s->arena->release(ob->off, ob->bytes);
        delete ob;
    }
    ob = nullptr;
}

// Launch of one admitted batch (without the mutex; the worker thread for
// persistent batches, a launcher thread for multi-kernel ones, whose sweep
// launches can block on a full launch queue).  Uses the slot's own handle.
bsvd_status launch_impl(bsvd_server_s* s, const Job& bt, int& cuda_err) {
    const int B = (int)bt.reqs.size();
    const Request* r0 = bt.reqs.front();
    const char t = r0->dtype;
    cudaStream_t st = bt.persistent ? s->streams[bt.slot] : s->streams_lo[bt.slot];
    std::vector<const void*> pA(B);
    std::vector<void*> pS(B), pU(B), pV(B);
    std::vector<int> mm(B), nn(B), lda(B), ldu(B), ldv(B);
    for (int i = 0; i < B; ++i) {
        const Request* r = bt.reqs[i];
        mm[i] = r->m; nn[i] = r->n; lda[i] = r->lda;
        ldu[i] = r->m; ldv[i] = r->n;
        pA[i] = r->A; pS[i] = r->S; pU[i] = r->U; pV[i] = r->V;
    }
    char* w = s->arena_base + bt.ws_off;
    const size_t pa = align256((size_t)B * sizeof(void*));
    void** dA = reinterpret_cast<void**>(w);
    void** dS = reinterpret_cast<void**>(w + pa);
    void** dU = reinterpret_cast<void**>(w + 2 * pa);
    void** dV = reinterpret_cast<void**>(w + 3 * pa);
    void* work = w + 4 * pa;
    const size_t work_bytes = bt.ws_bytes - 4 * pa;
    // pageable sources: each copy returns once its source is staged
    cudaError_t ce = cudaMemcpyAsync(dA, pA.data(), B * sizeof(void*), cudaMemcpyHostToDevice, st);
    if (ce == cudaSuccess) ce = cudaMemcpyAsync(dS, pS.data(), B * sizeof(void*), cudaMemcpyHostToDevice, st);
    if (ce == cudaSuccess) ce = cudaMemcpyAsync(dU, pU.data(), B * sizeof(void*), cudaMemcpyHostToDevice, st);
    if (ce == cudaSuccess) ce = cudaMemcpyAsync(dV, pV.data(), B * sizeof(void*), cudaMemcpyHostToDevice, st);
    if (ce != cudaSuccess) {
        cuda_err = (int)ce;
        return BSVD_ERR_CUDA;
    }
    int* df = s->dflags[bt.slot];
    const int MB = s->max_batch;
    const bsvd_opts o = batch_opts(s, r0, bt.persistent);
    const bsvd_job ju = r0->wantU ? BSVD_JOB_SOME : BSVD_JOB_NONE, jv = r0->wantV ? BSVD_JOB_SOME : BSVD_JOB_NONE;
    bsvd_status rc;
    bsvd_handle h = s->slot_h[bt.slot];
    if (bt.persistent) {
        rc = bsvd::persistent_with_flags(h, t, r0->wantU, r0->wantV, B, mm.data(), nn.data(), dA, lda.data(), dS,
                                         dU, ldu.data(), dV, ldv.data(), df, df + MB, df + 2 * MB, df + 3 * MB, work,
                                         work_bytes, &o, st);
    } else {
        switch (t) {
            case 's': rc = bsvd_sgesvj_batched(h, ju, jv, B, mm.data(), nn.data(), (const float* const*)dA,
                                               lda.data(), (float* const*)dS, (float* const*)dU, ldu.data(),
                                               (float* const*)dV, ldv.data(), df, df + MB, work, work_bytes, &o, st);
                      break;
            case 'd': rc = bsvd_dgesvj_batched(h, ju, jv, B, mm.data(), nn.data(), (const double* const*)dA,
                                               lda.data(), (double* const*)dS, (double* const*)dU, ldu.data(),
                                               (double* const*)dV, ldv.data(), df, df + MB, work, work_bytes, &o, st);
                      break;
            case 'c': rc = bsvd_cgesvj_batched(h, ju, jv, B, mm.data(), nn.data(), (const void* const*)dA,
                                               lda.data(), (float* const*)dS, (void* const*)dU, ldu.data(),
                                               (void* const*)dV, ldv.data(), df, df + MB, work, work_bytes, &o, st);
                      break;
            default:  rc = bsvd_zgesvj_batched(h, ju, jv, B, mm.data(), nn.data(), (const void* const*)dA,
                                               lda.data(), (double* const*)dS, (void* const*)dU, ldu.data(),
                                               (void* const*)dV, ldv.data(), df, df + MB, work, work_bytes, &o, st);
                      break;
        }
    }
    if (rc != BSVD_OK) {
        if (rc == BSVD_ERR_CUDA) cuda_err = bsvd_last_cuda(h);
        return rc;
    }
    ce = cudaEventRecord(s->events[bt.slot], st);
    cuda_err = (int)ce;
    return ce == cudaSuccess ? BSVD_OK : BSVD_ERR_CUDA;
}

// Launches and records the outcome in the slot's launch state (and, for a
// CUDA failure, the error code).
void launch(bsvd_server_s* s, const Job& bt) {
    int cuda_err = 0;
    const bsvd_status rc = launch_impl(s, bt, cuda_err);
    if (rc != BSVD_OK) {
        cudaGetLastError();
        cudaStreamSynchronize(bt.persistent ? s->streams[bt.slot] : s->streams_lo[bt.slot]);   // work already queued
        cudaGetLastError();
    }
    s->launch_cuda[bt.slot] = cuda_err;
    s->launch_state[bt.slot].store(rc == BSVD_OK ? 1 : (int)rc, std::memory_order_release);
}

int load_acquire(const int* p) { return __atomic_load_n(p, __ATOMIC_ACQUIRE); }
int load_relaxed(const int* p) { return __atomic_load_n(p, __ATOMIC_RELAXED); }

// Retires the requests whose flags are up, and whole batches whose event has
// completed.  Mutex held.
void poll_running(bsvd_server_s* s) {
    bool any = false;
    const int MB = s->max_batch;
    for (size_t bi = 0; bi < s->running.size();) {
        Batch& bt = s->running[bi];
        const int* hf = s->hflags[bt.slot];
        const int ls = s->launch_state[bt.slot].load(std::memory_order_acquire);
        if (ls == 0) { ++bi; continue; }                  // its launcher is still issuing work
        if (ls < 0) {
            if (bt.launcher.joinable()) bt.launcher.join();
            for (int i : bt.pending) {
                bt.reqs[i]->info = s->launch_cuda[bt.slot];     // the cudaError_t, if any
                complete(s, bt.reqs[i], ls);
                s->in_flight--;
            }
            any = true;
            s->arena->release(bt.ws_off, bt.ws_bytes);
            drop_out(s, bt.out);
            s->slot_busy[bt.slot] = false;
            s->running.erase(s->running.begin() + bi);
            continue;
        }
        if (bt.persistent) {
            size_t w = 0;
            for (size_t j = 0; j < bt.pending.size(); ++j) {
                const int i = bt.pending[j];
                if (load_acquire(hf + 2 * MB + i)) {
                    Request* r = bt.reqs[i];
                    r->info = load_relaxed(hf + i);
                    r->sweeps = load_relaxed(hf + MB + i);
                    complete(s, r, BSVD_OK);
                    s->in_flight--;
                    any = true;
                } else {
                    bt.pending[w++] = i;
                }
            }
            bt.pending.resize(w);
        }
        const cudaError_t q = cudaEventQuery(s->events[bt.slot]);
        if (q == cudaErrorNotReady) { ++bi; continue; }
        if (q != cudaSuccess) cudaGetLastError();
        for (int i : bt.pending) {
            Request* r = bt.reqs[i];
            r->info = load_relaxed(hf + i);
            r->sweeps = load_relaxed(hf + MB + i);
            // a persistent batch raises every flag unless it was told to stop
            int st = q == cudaSuccess ? BSVD_OK : BSVD_ERR_CUDA;
            if (st == BSVD_OK && bt.persistent && !load_acquire(hf + 2 * MB + i))
                st = s->slot_abort[bt.slot] ? BSVD_ERR_CANCELLED : BSVD_ERR_CUDA;
            complete(s, r, st);
            s->in_flight--;
            any = true;
        }
        if (bt.launcher.joinable()) bt.launcher.join();
        s->arena->release(bt.ws_off, bt.ws_bytes);
        drop_out(s, bt.out);
        s->slot_busy[bt.slot] = false;
        s->running.erase(s->running.begin() + bi);
    }
    if (any) s->cv_done.notify_all();
}

// Forms and launches batches while a stream and memory are free.  Mutex held
// on entry and exit (released around the launch).
void admit(bsvd_server_s* s, std::unique_lock<std::mutex>& lk) {
    for (;;) {
        int slot = -1;
        for (int k = 0; k < s->max_inflight; ++k)
            if (!s->slot_busy[k]) { slot = k; break; }
        if (slot < 0) return;
        int big_busy = 0;
        for (int k = 0; k < s->max_inflight; ++k) big_busy += s->slot_busy[k] && s->slot_big[k];
        // the key whose oldest request is the oldest of all; multi-kernel
        // batches (long, one request at low load) may not take every stream,
        // so small requests always find one
        auto best = s->queues.end();
        for (auto it = s->queues.begin(); it != s->queues.end(); ++it) {
            if (it->second.empty()) continue;
            if (std::get<3>(it->first) && big_busy >= s->big_cap) continue;
            if (best == s->queues.end()) { best = it; continue; }
            const Request* a = it->second.front();
            const Request* b = best->second.front();
            if (a->t_submit < b->t_submit || (a->t_submit == b->t_submit && a->id < b->id)) best = it;
        }
        if (best == s->queues.end()) return;
        std::deque<Request*>& q = best->second;
        Batch bt;
        bt.persistent = std::get<3>(best->first) == 0;
        bt.slot = slot;
        size_t take = std::min<size_t>(q.size(), (size_t)(bt.persistent ? s->max_batch : s->max_big_batch));
        bool fits = false, never = false;
        while (take > 0) {
            std::vector<Request*> rs(q.begin(), q.begin() + take);
            bt.ws_bytes = ws_bytes(s, s->h, rs, bt.persistent);
            size_t ob = 0;
            for (const Request* r : rs) ob += out_bytes(r);
            if (bt.ws_bytes == 0 ||
                (take == 1 && align256(bt.ws_bytes) + align256(ob) > s->arena->size())) {
                never = take == 1 || bt.ws_bytes == 0;
                break;
            }
            size_t off_out = 0;
            if (s->arena->alloc(bt.ws_bytes, bt.ws_off)) {
                if (s->arena->alloc(ob, off_out)) {
                    bt.reqs = rs;
                    bt.out = new OutBlock();
                    bt.out->off = off_out;
                    bt.out->bytes = ob;
                    fits = true;
                    break;
                }
                s->arena->release(bt.ws_off, bt.ws_bytes);
            }
            take /= 2;
        }
        if (!fits) {
            if (never) {
                // unplannable, or larger than the whole arena: fail the oldest request now
                Request* r = q.front();
                q.pop_front();
                s->queued--;
                complete(s, r, bt.ws_bytes == 0 ? BSVD_ERR_INVALID : BSVD_ERR_WORKSPACE);
                s->cv_done.notify_all();
                continue;
            }
            return;   // wait for memory, in arrival order
        }
        q.erase(q.begin(), q.begin() + bt.reqs.size());
        s->queued -= (long long)bt.reqs.size();
        s->in_flight += (long long)bt.reqs.size();
        bt.out->refs = (int)bt.reqs.size() + 1;
        char* o = s->arena_base + bt.out->off;
        size_t pos = 0;
        for (size_t i = 0; i < bt.reqs.size(); ++i) {
            Request* r = bt.reqs[i];
            const size_t e = elt_size(r->dtype);
            r->state = kRunning;
            r->out = bt.out;
            r->S = o + pos; pos += align256((size_t)r->k * real_size(r->dtype));
            if (r->wantU) { r->U = o + pos; pos += align256((size_t)r->m * r->k * e); }
            if (r->wantV) { r->V = o + pos; pos += align256((size_t)r->n * r->k * e); }
            bt.pending.push_back((int)i);
        }
        s->slot_busy[slot] = true;
        s->slot_big[slot] = !bt.persistent;
        s->slot_abort[slot] = false;
        std::memset(s->hflags[slot], 0, sizeof(int) * flag_ints(s));   // its previous batch has ended
        s->launched++;
        if (!bt.persistent) {
            s->launch_state[slot].store(0, std::memory_order_release);
            const Job job = bt;                          // what the launcher reads
            bt.launcher = std::thread([s, job]() {
                cudaSetDevice(s->device);
                launch(s, job);
                s->cv_work.notify_one();
            });
            s->running.push_back(std::move(bt));
            continue;
        }
        lk.unlock();
        launch(s, bt);
        lk.lock();
        s->running.push_back(std::move(bt));
    }
}

bool any_queued(const bsvd_server_s* s) {
    for (auto& kv : s->queues)
        if (!kv.second.empty()) return true;
    return false;
}

void worker_loop(bsvd_server_s* s) {
    cudaSetDevice(s->device);
    std::unique_lock<std::mutex> lk(s->mu);
    for (;;) {
        poll_running(s);
        if (!s->stop && !s->paused) admit(s, lk);
        if (s->stop && s->running.empty()) break;
        if (s->running.empty()) {
            // nothing runs: what is queued waits for memory (or was just
            // admitted), so sleep until a submit, release, pause or cancel
            // changes something -- never spin holding the mutex
            const long long g = s->wake_gen;
            s->cv_work.wait(lk, [&] { return s->stop || (!s->paused && any_queued(s) && s->wake_gen != g); });
        } else
            s->cv_work.wait_for(lk, std::chrono::microseconds(20));
    }
}

bsvd_status submit_at(bsvd_server_s* s, char dtype, int m, int n, const void* A, int lda, bsvd_job jobu,
                      bsvd_job jobv, double t_submit, long long* id) {
    if (!id) return BSVD_ERR_INVALID;
    if (dtype != 's' && dtype != 'd' && dtype != 'c' && dtype != 'z') return BSVD_ERR_INVALID;
    if (m < 1 || n < 1 || !A || lda < m) return BSVD_ERR_INVALID;
    if ((jobu != BSVD_JOB_NONE && jobu != BSVD_JOB_SOME) || (jobv != BSVD_JOB_NONE && jobv != BSVD_JOB_SOME))
        return BSVD_ERR_INVALID;
    cudaPointerAttributes at;
    if (cudaPointerGetAttributes(&at, A) != cudaSuccess) {
        cudaGetLastError();
        return BSVD_ERR_INVALID;
    }
    const void* dev = nullptr;
    if (at.type == cudaMemoryTypeDevice || at.type == cudaMemoryTypeManaged)
        dev = A;
    else if (at.type == cudaMemoryTypeHost && at.devicePointer)
        dev = at.devicePointer;
    if (!dev) return BSVD_ERR_INVALID;         // pageable host memory: the kernels cannot read it
    if (at.type == cudaMemoryTypeDevice && at.device != s->device) return BSVD_ERR_INVALID;
    Request* r = new (std::nothrow) Request();
    if (!r) return BSVD_ERR_NOMEM;
    r->dtype = dtype; r->m = m; r->n = n; r->k = std::min(m, n); r->lda = lda; r->A = dev;
    r->wantU = jobu == BSVD_JOB_SOME; r->wantV = jobv == BSVD_JOB_SOME;
    r->t_submit = t_submit;
    {
        std::lock_guard<std::mutex> lk(s->mu);
        if (s->stop) { delete r; return BSVD_ERR_INVALID; }
        r->id = s->next_id++;
        s->reqs[r->id] = r;
        s->queues[key_of(s, r)].push_back(r);
        s->submitted++;
        s->queued++;
        s->wake_gen++;
    }
    s->cv_work.notify_one();
    *id = r->id;
    return BSVD_OK;
}

// Queued requests complete as cancelled; busy slots get their abort flag.
void cancel_locked(bsvd_server_s* s) {
    for (auto& kv : s->queues) {
        for (Request* r : kv.second) {
            complete(s, r, BSVD_ERR_CANCELLED);
            s->queued--;
        }
        kv.second.clear();
    }
    for (int k = 0; k < s->max_inflight; ++k)
        if (s->slot_busy[k]) {
            s->slot_abort[k] = true;
            __atomic_store_n(s->hflags[k] + 3 * (size_t)s->max_batch, 1, __ATOMIC_RELEASE);
        }
}

int status_of(const Request* r) {
    return r->state == kDone ? 1 : r->state == kFailed ? r->status : 0;
}

bsvd_status release_locked(bsvd_server_s* s, std::map<long long, Request*>::iterator it) {
    Request* r = it->second;
    if (r->state != kDone && r->state != kFailed) return BSVD_ERR_INVALID;
    drop_out(s, r->out);
    s->reqs.erase(it);
    delete r;
    s->wake_gen++;
    return BSVD_OK;
}

}  // namespace

extern "C" {

double bsvd_server_clock(void) { return now_s(); }

bsvd_status bsvd_server_create(void* d_arena, size_t arena_bytes, const bsvd_server_opts* opts, bsvd_server* out) {
    if (!out) return BSVD_ERR_INVALID;
    *out = nullptr;
    if (!d_arena || arena_bytes < ((size_t)1 << 20) || (reinterpret_cast<uintptr_t>(d_arena) & 255))
        return BSVD_ERR_INVALID;
    bsvd_server_opts z;
    std::memset(&z, 0, sizeof z);
    if (!opts) opts = &z;
    if (opts->max_inflight < 0 || opts->max_inflight > 64 || opts->max_batch < 0 || opts->big_k < 0 ||
        opts->max_big_batch < 0 || (opts->fp64_prec != BSVD_PREC_NATIVE && opts->fp64_prec != BSVD_PREC_MIXED) ||
        opts->big_flags < 0 || opts->big_flags > 8191 || opts->big_k_fp64 < 0)
        return BSVD_ERR_INVALID;
    bsvd_server_s* s = new (std::nothrow) bsvd_server_s();
    if (!s) return BSVD_ERR_NOMEM;
    s->max_inflight = opts->max_inflight ? opts->max_inflight : 32;
    s->max_batch = opts->max_batch ? opts->max_batch : 4096;
    s->big_k = opts->big_k ? opts->big_k : 256;
    s->big_k_fp64 = opts->big_k_fp64 ? opts->big_k_fp64 : s->big_k;
    s->max_big_batch = opts->max_big_batch ? opts->max_big_batch : 8;
    s->fp64_prec = opts->fp64_prec;
    s->big_flags = opts->big_flags;
    s->arena_base = static_cast<char*>(d_arena);
    bsvd_status rc = BSVD_OK;
    if (cudaGetDevice(&s->device) != cudaSuccess) rc = BSVD_ERR_CUDA;
    if (rc == BSVD_OK) rc = bsvd_create(&s->h);
    if (rc == BSVD_OK) {
        s->arena = new (std::nothrow) Arena(arena_bytes);
        if (!s->arena) rc = BSVD_ERR_NOMEM;
    }
    s->streams.assign(s->max_inflight, nullptr);
    s->streams_lo.assign(s->max_inflight, nullptr);
    s->events.assign(s->max_inflight, nullptr);
    s->hflags.assign(s->max_inflight, nullptr);
    s->dflags.assign(s->max_inflight, nullptr);
    s->slot_busy.assign(s->max_inflight, false);
    s->slot_abort.assign(s->max_inflight, false);
    s->slot_big.assign(s->max_inflight, false);
    s->slot_h.assign(s->max_inflight, nullptr);
    s->launch_cuda.assign(s->max_inflight, 0);
    s->launch_state.reset(new (std::nothrow) std::atomic<int>[s->max_inflight]);
    if (!s->launch_state) rc = BSVD_ERR_NOMEM;
    for (int k = 0; k < s->max_inflight && rc == BSVD_OK; ++k) {
        s->launch_state[k].store(1);
        rc = bsvd_create(&s->slot_h[k]);
    }
    s->big_cap = std::max(1, s->max_inflight - std::max(2, s->max_inflight / 4));
    for (int k = 0; k < s->max_inflight && rc == BSVD_OK; ++k) {
        void* hp = nullptr;
        void* dp = nullptr;
        int lo = 0, hi = 0;
        if (cudaDeviceGetStreamPriorityRange(&lo, &hi) != cudaSuccess ||
            cudaStreamCreateWithPriority(&s->streams[k], cudaStreamNonBlocking, hi) != cudaSuccess ||
            cudaStreamCreateWithPriority(&s->streams_lo[k], cudaStreamNonBlocking, lo) != cudaSuccess ||
            cudaEventCreateWithFlags(&s->events[k], cudaEventDisableTiming) != cudaSuccess ||
            cudaHostAlloc(&hp, sizeof(int) * flag_ints(s), cudaHostAllocMapped) != cudaSuccess) {
            rc = BSVD_ERR_CUDA;
            break;
        }
        s->hflags[k] = static_cast<int*>(hp);
        if (cudaHostGetDevicePointer(&dp, hp, 0) != cudaSuccess) { rc = BSVD_ERR_CUDA; break; }
        s->dflags[k] = static_cast<int*>(dp);
        std::memset(hp, 0, sizeof(int) * flag_ints(s));
    }
    if (rc == BSVD_OK && cudaStreamCreateWithFlags(&s->fetch_stream, cudaStreamNonBlocking) != cudaSuccess)
        rc = BSVD_ERR_CUDA;
    if (rc != BSVD_OK) {
        cudaGetLastError();
        for (int k = 0; k < s->max_inflight; ++k) {
            if (s->streams[k]) cudaStreamDestroy(s->streams[k]);
            if (s->streams_lo[k]) cudaStreamDestroy(s->streams_lo[k]);
            if (s->events[k]) cudaEventDestroy(s->events[k]);
            if (s->hflags[k]) cudaFreeHost(s->hflags[k]);
        }
        if (s->fetch_stream) cudaStreamDestroy(s->fetch_stream);
        for (bsvd_handle hh : s->slot_h)
            if (hh) bsvd_destroy(hh);
        if (s->h) bsvd_destroy(s->h);
        delete s->arena;
        delete s;
        return rc;
    }
    s->worker = std::thread(worker_loop, s);
    *out = s;
    return BSVD_OK;
}

bsvd_status bsvd_server_submit(bsvd_server s, char dtype, int m, int n, const void* A, int lda, bsvd_job jobu,
                               bsvd_job jobv, long long* id) {
    if (!s) return BSVD_ERR_INVALID;
    return submit_at(s, dtype, m, n, A, lda, jobu, jobv, now_s(), id);
}

bsvd_status bsvd_server_replay(bsvd_server s, int count, const double* t_offset, const char* dtype, const int* m,
                               const int* n, const void* const* A, const int* lda, bsvd_job jobu, bsvd_job jobv,
                               long long* ids, double* t0) {
    if (!s || count < 0 || (count > 0 && (!t_offset || !dtype || !m || !n || !A || !lda || !ids)))
        return BSVD_ERR_INVALID;
    const double start = now_s();
    if (t0) *t0 = start;
    for (int i = 0; i < count; ++i) {
        const double target = start + t_offset[i];
        for (;;) {
            const double left = target - now_s();
            if (left <= 0) break;
            if (left > 300e-6) std::this_thread::sleep_for(std::chrono::duration<double>(left - 200e-6));
        }
        const bsvd_status rc = submit_at(s, dtype[i], m[i], n[i], A[i], lda[i], jobu, jobv, target, &ids[i]);
        if (rc != BSVD_OK) return rc;
    }
    return BSVD_OK;
}

int bsvd_server_test(bsvd_server s, long long id) {
    if (!s) return BSVD_ERR_INVALID;
    std::lock_guard<std::mutex> lk(s->mu);
    auto it = s->reqs.find(id);
    if (it == s->reqs.end()) return BSVD_ERR_INVALID;
    return status_of(it->second);
}

bsvd_status bsvd_server_wait(bsvd_server s, long long id, double timeout_s, int* info, int* sweeps, double* t_done) {
    if (!s) return BSVD_ERR_INVALID;
    std::unique_lock<std::mutex> lk(s->mu);
    auto it = s->reqs.find(id);
    if (it == s->reqs.end()) return BSVD_ERR_INVALID;
    Request* r = it->second;
    auto ready = [&] { return r->state == kDone || r->state == kFailed; };
    if (timeout_s < 0) s->cv_done.wait(lk, ready);
    else if (!s->cv_done.wait_for(lk, std::chrono::duration<double>(timeout_s), ready)) return BSVD_ERR_TIMEOUT;
    if (info) *info = r->info;
    if (sweeps) *sweeps = r->sweeps;
    if (t_done) *t_done = r->t_done;
    return r->state == kDone ? BSVD_OK : (bsvd_status)r->status;
}

bsvd_status bsvd_server_result(bsvd_server s, long long id, void** dS, void** dU, int* ldu, void** dV, int* ldv) {
    if (!s) return BSVD_ERR_INVALID;
    std::lock_guard<std::mutex> lk(s->mu);
    auto it = s->reqs.find(id);
    if (it == s->reqs.end() || it->second->state != kDone) return BSVD_ERR_INVALID;
    const Request* r = it->second;
    if (dS) *dS = r->S;
    if (dU) *dU = r->U;
    if (ldu) *ldu = r->m;
    if (dV) *dV = r->V;
    if (ldv) *ldv = r->n;
    return BSVD_OK;
}

bsvd_status bsvd_server_fetch(bsvd_server s, long long id, void* S, void* U, int ldu, void* V, int ldv) {
    if (!s) return BSVD_ERR_INVALID;
    Request r;
    {
        std::lock_guard<std::mutex> lk(s->mu);
        auto it = s->reqs.find(id);
        if (it == s->reqs.end() || it->second->state != kDone) return BSVD_ERR_INVALID;
        r = *it->second;
    }
    if ((U && (!r.U || ldu < r.m)) || (V && (!r.V || ldv < r.n))) return BSVD_ERR_INVALID;
    int prev = -1;
    cudaGetDevice(&prev);
    if (prev != s->device) cudaSetDevice(s->device);
    const size_t e = elt_size(r.dtype);
    cudaError_t ce = cudaSuccess;
    if (S) ce = cudaMemcpyAsync(S, r.S, (size_t)r.k * real_size(r.dtype), cudaMemcpyDefault, s->fetch_stream);
    if (ce == cudaSuccess && U)
        ce = cudaMemcpy2DAsync(U, (size_t)ldu * e, r.U, (size_t)r.m * e, (size_t)r.m * e, r.k, cudaMemcpyDefault,
                               s->fetch_stream);
    if (ce == cudaSuccess && V)
        ce = cudaMemcpy2DAsync(V, (size_t)ldv * e, r.V, (size_t)r.n * e, (size_t)r.n * e, r.k, cudaMemcpyDefault,
                               s->fetch_stream);
    const cudaError_t se = cudaStreamSynchronize(s->fetch_stream);
    if (prev >= 0 && prev != s->device) cudaSetDevice(prev);
    if (ce != cudaSuccess || se != cudaSuccess) {
        cudaGetLastError();
        return BSVD_ERR_CUDA;
    }
    return BSVD_OK;
}

bsvd_status bsvd_server_release(bsvd_server s, long long id) {
    if (!s) return BSVD_ERR_INVALID;
    bsvd_status rc;
    {
        std::lock_guard<std::mutex> lk(s->mu);
        auto it = s->reqs.find(id);
        if (it == s->reqs.end()) return BSVD_ERR_INVALID;
        rc = release_locked(s, it);
    }
    if (rc == BSVD_OK) s->cv_work.notify_one();      // freed memory may admit a waiting batch
    return rc;
}

int bsvd_server_collect(bsvd_server s, int max, int release, long long* ids, int* status, int* info, int* sweeps,
                        double* t_submit, double* t_done) {
    if (!s || max < 0) return BSVD_ERR_INVALID;
    int k = 0;
    bool freed = false;
    {
        std::lock_guard<std::mutex> lk(s->mu);
        while (k < max && !s->completions.empty()) {
            const long long id = s->completions.front();
            s->completions.pop_front();
            auto it = s->reqs.find(id);
            if (it == s->reqs.end()) continue;           // released already
            const Request* r = it->second;
            if (ids) ids[k] = id;
            if (status) status[k] = r->state == kDone ? 0 : r->status;
            if (info) info[k] = r->info;
            if (sweeps) sweeps[k] = r->sweeps;
            if (t_submit) t_submit[k] = r->t_submit;
            if (t_done) t_done[k] = r->t_done;
            ++k;
            if (release) {
                release_locked(s, it);
                freed = true;
            }
        }
    }
    if (freed) s->cv_work.notify_one();
    return k;
}

bsvd_status bsvd_server_cancel(bsvd_server s) {
    if (!s) return BSVD_ERR_INVALID;
    {
        std::lock_guard<std::mutex> lk(s->mu);
        cancel_locked(s);
    }
    s->cv_done.notify_all();
    return BSVD_OK;
}

bsvd_status bsvd_server_pause(bsvd_server s, int paused) {
    if (!s) return BSVD_ERR_INVALID;
    {
        std::lock_guard<std::mutex> lk(s->mu);
        s->paused = paused != 0;
        s->wake_gen++;
    }
    s->cv_work.notify_one();
    return BSVD_OK;
}

bsvd_status bsvd_server_stats(bsvd_server s, long long* c) {
    if (!s || !c) return BSVD_ERR_INVALID;
    std::lock_guard<std::mutex> lk(s->mu);
    c[0] = s->submitted;
    c[1] = s->completed;
    c[2] = s->failed;
    c[3] = s->queued;
    c[4] = s->in_flight;
    c[5] = (long long)s->running.size();
    c[6] = (long long)s->arena->used();
    c[7] = (long long)s->arena->peak();
    c[8] = s->cancelled;
    c[9] = s->launched;
    return BSVD_OK;
}

bsvd_status bsvd_server_destroy(bsvd_server s) {
    if (!s) return BSVD_ERR_INVALID;
    {
        std::lock_guard<std::mutex> lk(s->mu);
        s->stop = true;
        cancel_locked(s);
    }
    s->cv_work.notify_all();
    s->cv_done.notify_all();
    if (s->worker.joinable()) s->worker.join();   // returns once the running batches have ended
    for (auto& kv : s->reqs) delete kv.second;
    for (int k = 0; k < s->max_inflight; ++k) {
        if (s->streams[k]) cudaStreamDestroy(s->streams[k]);
        if (s->streams_lo[k]) cudaStreamDestroy(s->streams_lo[k]);
        if (s->events[k]) cudaEventDestroy(s->events[k]);
        if (s->hflags[k]) cudaFreeHost(s->hflags[k]);
    }
    if (s->fetch_stream) cudaStreamDestroy(s->fetch_stream);
    for (bsvd_handle hh : s->slot_h) bsvd_destroy(hh);
    bsvd_destroy(s->h);
    delete s->arena;
    delete s;
    return BSVD_OK;
}

}  // extern "C"
