// C ABI of libdfs (declared in include/dfs.h): argument checks, workspace planning and the
// launch sequence of Algorithm 1 (arXiv 2310.17556) with Q inlined (Section 2).
#include <cmath>
#include <algorithm>
#include <array>
#include <cstdarg>
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <string>
#include <vector>

#include "kernels.cuh"

using namespace dfs;

namespace dfs {
std::atomic<long long>& launch_counter() {
    static std::atomic<long long> c{0};
    return c;
}
}  // namespace dfs

struct dfs_handle_s {
    int device = 0;
    int num_sms = 0;
    size_t smem_optin = 0;
    void* ws = nullptr;
    size_t ws_bytes = 0;
    DevStatus* dstat = nullptr;
    void* hbuf[3] = {nullptr, nullptr, nullptr};  // device staging (dfs_solve_host, dfs_solve_complex): S, V, X
    int* bstat = nullptr;                          // per-problem device status of dfs_solve_batched
    int bstat_count = 0;
    int bstat_used = 0;                            // problems of the last dfs_solve_batched
    // dfs_solve_batched runs its problems on up to kMaxLanes concurrent lanes: each a private handle
    // (workspace, device status) and stream, forked from and joined to the caller's stream by events.
    static constexpr int kMaxLanes = 16;
    int batch_lanes = 8;  // lanes dfs_solve_batched uses (dfs_autotune_batched may change it)
    int batch_share = 1;  // each lane's kernels take 1 / batch_share of the SMs (grid sizes)
    dfs_handle lane[kMaxLanes] = {};
    cudaStream_t lane_stream[kMaxLanes] = {};
    cudaEvent_t lane_done[kMaxLanes] = {};
    cudaEvent_t fork_ev = nullptr;
    int chol_share = 1;  // the cooperative Cholesky takes 1 / chol_share of the resident-CTA capacity
    bool lane_handle = false;  // a lane of dfs_solve_batched: no whole-GPU fused Gram (lanes run concurrently)
    int test_fault = 0;                    // dfs_set_test_fault: DFS_TEST_FAULT_* for the next calls
    unsigned long long test_wait_ns = 0;   // and the limit of their device waits (0: the default)
    // dfs_solve_host_async: two device staging slots for S and V (alternating calls), one for X, a
    // copy stream for the uploads and the events that order slot reuse
    void* abuf[2][2] = {{nullptr, nullptr}, {nullptr, nullptr}};
    size_t abuf_bytes[2][2] = {{0, 0}, {0, 0}};
    void* axbuf = nullptr;
    size_t axbuf_bytes = 0;
    cudaStream_t copy_stream = nullptr;
    cudaEvent_t slot_free[2] = {nullptr, nullptr};
    cudaEvent_t slot_copied[2] = {nullptr, nullptr};
    bool slot_used[2] = {false, false};
    int aslot = 0;
    size_t hbuf_bytes[3] = {0, 0, 0};
    int last_precision = 0;
    // Step-timing events: a ring of kTimingSlots solves x kMarks marks (DFS_FLAG_STEP_TIMING).
    // Marks: 0 start, 1 Gram kernel start, 2 Gram kernel end, 3 Cholesky end, 4 first n-space
    // solve end, 5 end of the call.
    static constexpr int kTimingSlots = 64;
    static constexpr int kMarks = 13;
    cudaEvent_t ev[kTimingSlots][kMarks] = {};
    int tslot = 0;      // slot of the last timed solve
    int tpending = 0;   // timed solves not yet summarised by dfs_step_times
    bool timed = false;  // last solve recorded the step events
    std::string err;
};

namespace {

constexpr size_t kAlign = 256;

size_t align_up(size_t x) { return (x + kAlign - 1) / kAlign * kAlign; }

int elem_size(int dt) { return dt == DFS_F64 ? 8 : (dt == DFS_F32 ? 4 : 2); }

// Records the message on the handle; with DFS_LOG set in the environment (to anything but "0")
// also prints it to stderr.  The library prints nothing otherwise.
dfs_status fail(dfs_handle h, dfs_status s, const char* fmt, ...) {
    char buf[512];
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(buf, sizeof(buf), fmt, ap);
    va_end(ap);
    if (h) h->err = buf;
    static const bool log = [] {
        const char* e = std::getenv("DFS_LOG");
        return e != nullptr && std::strcmp(e, "0") != 0;
    }();
    if (log) std::fprintf(stderr, "dfs: %s: %s\n", dfs_status_string(s), buf);
    return s;
}

#define DFS_CK(call)                                                                       \
    do {                                                                                   \
        cudaError_t e_ = (call);                                                           \
        if (e_ != cudaSuccess)                                                             \
            return fail(h, DFS_ERR_CUDA, "%s failed: %s (%s:%d)", #call, cudaGetErrorString(e_), \
                        __FILE__, __LINE__);                                               \
    } while (0)

struct Plan {
    int s_dtype = DFS_F32;
    int prec = DFS_PREC_FP32;
    bool f64 = false;     // n-space solve type is FP64
    bool tensor = false;  // tcgen05 Gram + refinement
    int64_t n = 0, m = 0, n_pad = 0;
    int k = 1, kq = 1;
    int nsplit = 1;
    int64_t chunk = 0;
    GramTcPlan tc{};
    PassPlan pp{};
    int pgrid = 1;  // rows of the pass partial buffers
    int pack = 0;   // tile packing done by the first S v pass: 0 none, 1 BF16, 2 TF32
    bool fused = false;  // b = S v, the BF16 tiles and the Gram in one kernel (gram_fused.cu)
    bool ns = false;  // n-space steps as one cluster kernel (nspace.cu)
    size_t off_W = 0, off_Linv = 0, off_P = 0, off_Rpart = 0, off_U2part = 0, off_R = 0, off_Z = 0, off_Y = 0,
           off_U2 = 0, off_V = 0, off_bn2 = 0, off_Sp = 0, off_Cf = 0, off_Rs = 0, off_Yc = 0, off_Cg = 0,
           off_Rdy = 0, total = 0;
};

int tc_kind(int prec) {
    switch (prec) {
        case DFS_PREC_BF16: return 0;
        case DFS_PREC_TF32: return 1;
        case DFS_PREC_BF16X3: return 2;
        case DFS_PREC_FP8: return 3;
        default: return -1;
    }
}

dfs_status resolve_precision(dfs_handle h, int s_dtype, int prec, int* out) {
    if (prec == DFS_PREC_AUTO) {
        if (s_dtype == DFS_F64) prec = DFS_PREC_FP64;
        else if (gram_tc_supported(s_dtype, 0)) prec = DFS_PREC_BF16;
        else if (gram_tc_supported(s_dtype, 1)) prec = DFS_PREC_TF32;
        else prec = DFS_PREC_FP32;
    }
    switch (prec) {
        case DFS_PREC_FP64:
            if (s_dtype != DFS_F64) return fail(h, DFS_ERR_INVALID_ARG, "precision FP64 needs FP64 S");
            break;
        case DFS_PREC_FP32:
            if (s_dtype == DFS_F64) return fail(h, DFS_ERR_INVALID_ARG, "precision FP32 needs FP32 or BF16 S");
            break;
        case DFS_PREC_BF16:
        case DFS_PREC_TF32:
        case DFS_PREC_BF16X3:
        case DFS_PREC_FP8:
            if (!gram_tc_supported(s_dtype, tc_kind(prec)))
                return fail(h, DFS_ERR_UNSUPPORTED, "tensor-core Gram kind %d not available for S dtype %d",
                            tc_kind(prec), s_dtype);
            break;
        default:
            return fail(h, DFS_ERR_INVALID_ARG, "unknown precision %d", prec);
    }
    *out = prec;
    return DFS_OK;
}

int pow2_at_least(int k) {
    int q = 1;
    while (q < k && q < 8) q <<= 1;
    return q;
}

// kq_cap > 0: at most that many right-hand sides per group (DFS_FLAG_RHS_GROUP, or the tuner's
// choice); 0 = as many as the kernels take
dfs_status make_plan(dfs_handle h, int s_dtype, int prec, int64_t n, int64_t m, int k, Plan* p,
                     bool allow_fused = true, int kq_cap = 0) {
    p->s_dtype = s_dtype;
    p->prec = prec;
    p->f64 = (prec == DFS_PREC_FP64);
    p->tensor = tc_kind(prec) >= 0;
    p->n = n;
    p->m = m;
    p->n_pad = round_up(n, 128);
    p->k = k;
    const int es = p->f64 ? 8 : 4;
    int kq = pow2_at_least(k);
    if (kq_cap > 0 && kq > kq_cap) kq = pow2_at_least(kq_cap);
    int kq_pass = pass_max_group((int)n, s_dtype, h->smem_optin);
    // the cluster pass (FP32 S, n <= 4096) keeps its rows in registers: it takes up to 8 right-hand
    // sides (n <= 2048) whatever the one-CTA-per-strip pass's shared-memory bound is
    for (int c = 8; c > kq_pass; c >>= 1) {
        int cs = 0, crpt = 0;
        if (pass_cluster_plan(s_dtype, (int)n, c, h->num_sms, m, h->smem_optin, &cs, &crpt) > 0) {
            kq_pass = c;
            break;
        }
    }
    const int kq_trsv = trsv_max_group((int)p->n_pad, es, h->smem_optin);
    if (kq_pass < 1 || kq_trsv < 1)
        return fail(h, DFS_ERR_UNSUPPORTED, "n=%lld too large for the on-chip n-space buffers", (long long)n);
    if (kq > kq_pass) kq = kq_pass;
    if (kq > kq_trsv) kq = kq_trsv;
    p->kq = kq;
    size_t gram_bytes;
    if (p->tensor) {
        p->tc = gram_tc_plan(s_dtype, tc_kind(prec), n, m, h->num_sms);
        GramTcPlan fp;
        if (tc_kind(prec) == 0 && allow_fused && !h->lane_handle &&
            gram_fused_plan(s_dtype, n, m, kq, h->num_sms, h->smem_optin, &fp)) {
            p->tc = fp;
            p->fused = true;
        }
        gram_bytes = p->tc.partial_bytes;
    } else {
        gram_simt_plan(n, m, p->f64, h->num_sms, &p->nsplit, &p->chunk);
        gram_bytes = gram_simt_partial_bytes(n, p->f64, p->nsplit);
    }
    p->pp = pass_make_plan((int)n, kq, s_dtype, h->num_sms, m, h->smem_optin);
    p->pgrid = pass_partial_rows(p->pp);
    if (p->fused && p->pgrid < h->num_sms) p->pgrid = h->num_sms;  // the fused kernel's row sums: one row per CTA
    p->pack = (p->tensor && p->tc.packed) ? (p->tc.kind == 1 ? 2 : (p->tc.kind == 2 ? 3 : (p->tc.kind == 3 ? 4 : 1)))
                                          : 0;
    p->ns = nspace_slots((int)p->n_pad, kq, (int)es, h->smem_optin) >= 2;
    size_t off = 0;
    auto take = [&](size_t bytes) {
        const size_t o = off;
        off = align_up(off + bytes);
        return o;
    };
    const size_t np = (size_t)p->n_pad;
    p->off_W = take(np * np * es);
    p->off_Linv = take(np * 32 * es);
    p->off_P = take(gram_bytes);
    p->off_Rpart = take((size_t)p->pgrid * n * kq * 8);
    p->off_U2part = take((size_t)std::max(p->pgrid, tile_correct_parts(h->num_sms)) * 2 * kq * 8);
    p->off_R = take(np * kq * 8);
    p->off_Z = take(np * kq * es);
    p->off_Y = take(np * kq * 8);
    p->off_U2 = take(16 * 8);
    p->off_V = take(p->tensor ? (size_t)k * round_up(m, 4) * (p->f64 ? 8 : 4) : 0);
    p->off_bn2 = take(8 * 8);
    p->off_Sp = take(pack_bytes(s_dtype, p->pack, n, m));
    p->off_Cf = take(cholesky_flag_bytes(p->n_pad));
    p->off_Rs = take(p->pack == 4 ? 2 * np * sizeof(float) : 0);
    p->off_Yc = take(np * kq * 8);  // centred scores: P y / sqrt(n) for the passes
    p->off_Cg = take(center_gram_scratch_doubles(np) * 8);
    p->off_Rdy = take(p->fused ? gram_fused_ready_bytes(p->tc) : 0);
    p->total = off;
    return DFS_OK;
}

dfs_status ensure_ws(dfs_handle h, size_t bytes, cudaStream_t stream) {
    if (bytes <= h->ws_bytes) return DFS_OK;
    cudaStreamCaptureStatus cs = cudaStreamCaptureStatusNone;
    if (cudaStreamIsCapturing(stream, &cs) == cudaSuccess && cs != cudaStreamCaptureStatusNone)
        return fail(h, DFS_ERR_NO_MEMORY, "workspace must grow to %zu bytes during stream capture; call dfs_reserve first",
                    bytes);
    if (h->ws) {
        cudaFree(h->ws);
        h->ws = nullptr;
        h->ws_bytes = 0;
    }
    if (cudaMalloc(&h->ws, bytes) != cudaSuccess) {
        cudaGetLastError();
        return fail(h, DFS_ERR_NO_MEMORY, "cudaMalloc(%zu) for the workspace failed", bytes);
    }
    h->ws_bytes = bytes;
    return DFS_OK;
}

template <typename P>
P* at(dfs_handle h, size_t off) {
    return reinterpret_cast<P*>(static_cast<char*>(h->ws) + off);
}

dfs_status check_s(dfs_handle h, const void* S, int s_dtype, int64_t n, int64_t m, int64_t lds) {
    if (s_dtype != DFS_F64 && s_dtype != DFS_F32 && s_dtype != DFS_BF16)
        return fail(h, DFS_ERR_INVALID_ARG, "unknown S dtype %d", s_dtype);
    if (!S) return fail(h, DFS_ERR_INVALID_ARG, "S is NULL");
    if (n < 1 || m < 1) return fail(h, DFS_ERR_INVALID_ARG, "n=%lld m=%lld must be >= 1", (long long)n, (long long)m);
    if (n > 65536) return fail(h, DFS_ERR_UNSUPPORTED, "n=%lld above the supported maximum 65536", (long long)n);
    if (lds < m) return fail(h, DFS_ERR_INVALID_ARG, "lds=%lld < m=%lld", (long long)lds, (long long)m);
    if (reinterpret_cast<uintptr_t>(S) % 16 != 0) return fail(h, DFS_ERR_INVALID_ARG, "S is not 16-byte aligned");
    if ((lds * elem_size(s_dtype)) % 16 != 0)
        return fail(h, DFS_ERR_INVALID_ARG, "lds * sizeof(S element) must be a multiple of 16 bytes");
    return DFS_OK;
}

dfs_status check_lambda(dfs_handle h, double lambda) {
    if (!std::isfinite(lambda) || !(lambda > 0.0))
        return fail(h, DFS_ERR_INVALID_ARG, "lambda must be finite and > 0 (got %g)", lambda);
    return DFS_OK;
}

// The Gram into W (rows < n_out, stride ldw): Gram + lambda on the diagonal (identity padding).
// The tensor-core Gram on packed tiles first runs the S v pass in packing mode (with no V).
dfs_status run_gram(dfs_handle h, const Plan& p, const void* S, int64_t lds, double lambda, void* W, int64_t ldw,
                    int64_t n_out, cudaStream_t stream) {
    void* P = at<void>(h, p.off_P);
    if (p.tensor) {
        void* Sp = p.pack ? at<void>(h, p.off_Sp) : nullptr;
        float* rs = p.pack == 4 ? at<float>(h, p.off_Rs) : nullptr;  // FP8 row scales, then their inverses
        if (rs) DFS_CK(launch_row_scale(p.s_dtype, S, (int)p.n, (int)p.n_pad, p.m, lds, rs, h->dstat, stream));
        if (p.fused) {
            DFS_CK(launch_gram_fused(p.tc, 1, S, p.n, p.m, lds, nullptr, p.m, 0, at<double>(h, p.off_Rpart), Sp, P,
                                     at<int>(h, p.off_Rdy), h->dstat, h->num_sms, stream, nullptr));
        } else {
            if (p.pack)
                DFS_CK(launch_sv_pack(p.pp, p.s_dtype, 1, p.pack, S, (int)p.n, p.m, lds, nullptr, p.m, 0,
                                      at<double>(h, p.off_Rpart), Sp, h->dstat, stream, rs ? rs + p.n_pad : nullptr));
            DFS_CK(launch_gram_tc(p.tc, p.s_dtype, S, p.n, p.m, lds, Sp, P, h->dstat, stream));
        }
        DFS_CK(launch_gram_tc_finalize(p.tc, P, p.n, n_out, lambda, W, ldw, stream, rs));
    } else {
        DFS_CK(launch_gram_simt(p.s_dtype, p.f64, S, p.n, p.m, lds, p.nsplit, p.chunk, P, stream));
        DFS_CK(launch_gram_finalize(p.f64, p.f64, gram_simt_tile(p.f64), P, p.nsplit, p.n, n_out, lambda, W, ldw,
                                    stream));
    }
    return DFS_OK;
}

// dfs_info.ms layout from the marks of one solve: 0 start, 1/2 around the Gram kernel, 3 after
// the Cholesky, 4 after the first triangular solves, 5 end, 6/7 around the S v pass, 8/9 around
// the first pass over S after the solves, 10 before the Cholesky kernel.
void step_ms(cudaEvent_t* e, float* ms) {
    float t[5];
    for (int i = 0; i < 5; ++i) cudaEventElapsedTime(&t[i], e[i], e[i + 1]);
    ms[0] = t[1];         // Gram kernel
    ms[1] = t[2];         // Gram finalize + Cholesky
    ms[2] = t[0] + t[3];  // S v pass (with tile packing) + first triangular solves
    ms[3] = t[4];         // refinement passes (or the x pass)
    cudaEventElapsedTime(&ms[4], e[0], e[5]);
    cudaEventElapsedTime(&ms[5], e[6], e[7]);   // S v pass kernel
    cudaEventElapsedTime(&ms[6], e[8], e[9]);   // first refinement (or x) pass kernel
    cudaEventElapsedTime(&ms[7], e[10], e[3]);  // Cholesky kernel
    cudaEventElapsedTime(&ms[8], e[11], e[12]);  // the correction from the packed tiles (0 if none)
}

dfs_status fill_info(dfs_handle h, cudaStream_t stream, dfs_info* info) {
    DevStatus ds;
    DFS_CK(cudaMemcpyAsync(&ds, h->dstat, sizeof(DevStatus), cudaMemcpyDeviceToHost, stream));
    DFS_CK(cudaStreamSynchronize(stream));
    if (info) {
        info->status = ds.status;
        info->precision_used = h->last_precision;
        info->iters = ds.iters;
        info->failed_pivot = ds.failed_pivot;
        info->passes = ds.passes;
        info->rel_correction = ds.rel_correction;
        info->rel_residual_n = ds.rel_residual;
        for (int i = 0; i < DFS_STEP_TIMES; ++i) info->ms[i] = 0.0f;
        if (h->timed) step_ms(h->ev[h->tslot], info->ms);
    }
    if (ds.status != 0) {
        if (ds.status == DFS_ERR_BOUNDS)
            return fail(h, DFS_ERR_BOUNDS, "device index check failed at source %d, line %d", ds.bounds_site / 100000,
                        ds.bounds_site % 100000);
        if (ds.status == DFS_ERR_NOT_SPD || ds.status == DFS_ERR_NONFINITE)
            return fail(h, (dfs_status)ds.status, "device reported %s at pivot %d", dfs_status_string(ds.status),
                        ds.failed_pivot);
        return fail(h, (dfs_status)ds.status, "device reported %s", dfs_status_string(ds.status));
    }
    return DFS_OK;
}

dfs_status solve_device(dfs_handle h, const void* S, int s_dtype, int64_t n, int64_t m, int64_t lds, const void* V,
                        int64_t k, int64_t ldv, double lambda, void* X, int64_t ldx, const dfs_options* opt,
                        cudaStream_t stream, dfs_info* info) {
    dfs_status s;
    if ((s = check_s(h, S, s_dtype, n, m, lds)) != DFS_OK) return s;
    if ((s = check_lambda(h, lambda)) != DFS_OK) return s;
    if (!V || !X) return fail(h, DFS_ERR_INVALID_ARG, "V or X is NULL");
    if (k < 1) return fail(h, DFS_ERR_INVALID_ARG, "k must be >= 1");
    if (ldv < m || ldx < m) return fail(h, DFS_ERR_INVALID_ARG, "ldv and ldx must be >= m");
    {
        const size_t es = s_dtype == DFS_F64 ? 8 : 4;
        const char* x0 = static_cast<const char*>(X);
        const char* x1 = x0 + ((k - 1) * ldx + m) * es;
        const char* s0 = static_cast<const char*>(S);
        const char* s1 = s0 + ((n - 1) * lds + m) * elem_size(s_dtype);
        if (x0 < s1 && s0 < x1) return fail(h, DFS_ERR_INVALID_ARG, "X overlaps S");
    }
    int prec;
    if ((s = resolve_precision(h, s_dtype, opt ? opt->precision : DFS_PREC_AUTO, &prec)) != DFS_OK) return s;
    const int max_iter = (opt && opt->max_iter >= 0) ? opt->max_iter : 8;
    const double tol = (opt && opt->tol > 0.0) ? opt->tol : 1e-7;
    Plan p;
    const bool allow_fused = !(opt && (opt->flags & DFS_FLAG_TWO_KERNEL_GRAM));
    const int kq_cap = opt ? (opt->flags >> 8) & 15 : 0;
    if ((s = make_plan(h, s_dtype, prec, n, m, (int)k, &p, allow_fused, kq_cap)) != DFS_OK) return s;
    if ((s = ensure_ws(h, p.total, stream)) != DFS_OK) return s;
    h->last_precision = prec;
    // S = (O - O_bar) / sqrt(n) from the caller's O: n-space centring around unchanged passes over
    // O (center.cu), on the reduce + triangular-solve kernels
    const bool center = opt && (opt->flags & DFS_FLAG_CENTER);
    if (center) p.ns = false;

    void* W = at<void>(h, p.off_W);
    void* Linv = at<void>(h, p.off_Linv);
    double* Rpart = at<double>(h, p.off_Rpart);
    double* U2part = at<double>(h, p.off_U2part);
    double* R = at<double>(h, p.off_R);
    void* Z = at<void>(h, p.off_Z);
    double* Y = at<double>(h, p.off_Y);
    double* U2 = at<double>(h, p.off_U2);
    double* bn2 = at<double>(h, p.off_bn2);
    double* Yc = at<double>(h, p.off_Yc);
    double* Yp = center ? Yc : Y;  // the y the passes read
    const int ni = (int)n, npi = (int)p.n_pad, kq = p.kq;
    const size_t vs = s_dtype == DFS_F64 ? 8 : 4;

    const bool timed = opt && (opt->flags & DFS_FLAG_STEP_TIMING);
    h->timed = false;
    int slot = 0;
    if (timed) {
        slot = (h->tslot + 1) % dfs_handle_s::kTimingSlots;
        if (!h->ev[slot][0])
            for (int i = 0; i < dfs_handle_s::kMarks; ++i) DFS_CK(cudaEventCreate(&h->ev[slot][i]));
    }
    cudaStreamCaptureStatus cap_status = cudaStreamCaptureStatusNone;
    if (cudaStreamIsCapturing(stream, &cap_status) != cudaSuccess) cudaGetLastError();
    const bool capturing = cap_status == cudaStreamCaptureStatusActive;
    auto mark = [&](int i) -> cudaError_t {
        // inside a stream capture the marks must be external event nodes, so that every replay of
        // the graph records them
        return timed ? cudaEventRecordWithFlags(h->ev[slot][i], stream,
                                                capturing ? cudaEventRecordExternal : cudaEventRecordDefault)
                     : cudaSuccess;
    };
    const int fp64_panel = opt && (opt->flags & DFS_FLAG_FP64_PANEL);

    if (p.tensor) {
        // Refinement reads V in every pass: when X overlaps V, work from a private copy of V.
        const char* v0 = static_cast<const char*>(V);
        const char* v1 = v0 + ((k - 1) * ldv + m) * vs;
        const char* x0 = static_cast<const char*>(X);
        const char* x1 = x0 + ((k - 1) * ldx + m) * vs;
        if (x0 < v1 && v0 < x1) {
            const int64_t ldc = round_up(m, 4);
            void* Vc = at<void>(h, p.off_V);
            DFS_CK(cudaMemcpy2DAsync(Vc, ldc * vs, V, ldv * vs, m * vs, k, cudaMemcpyDeviceToDevice, stream));
            V = Vc;
            ldv = ldc;
        }
    }
    void* Sp = p.pack ? at<void>(h, p.off_Sp) : nullptr;
    float* rs = p.pack == 4 ? at<float>(h, p.off_Rs) : nullptr;  // FP8 row scales, then their inverses

    DFS_CK(launch_status_reset(h->dstat, stream, h->test_wait_ns, h->test_fault));
    DFS_CK(mark(0));
    DFS_CK(mark(11));  // both re-recorded around the tile correction when it runs, else 0 ms apart
    DFS_CK(mark(12));
    if (rs) DFS_CK(launch_row_scale(s_dtype, S, (int)ni, (int)p.n_pad, m, lds, rs, h->dstat, stream));
    for (int64_t q0 = 0; q0 < k; q0 += kq) {
        const int kg = (int)((k - q0) < kq ? (k - q0) : kq);
        const void* Vg = static_cast<const char*>(V) + q0 * ldv * vs;
        void* Xg = static_cast<char*>(X) + q0 * ldx * vs;
        DFS_CK(launch_group_reset(h->dstat, stream));
        // b = S v; the first group's pass also writes the packed tensor-core tiles of S, and in the
        // fused form computes the Gram partials of Algorithm 1 step 1 in the same kernel
        const bool fused_now = q0 == 0 && p.fused;
        // (step marks: 6/7 around the S v pass, empty in the fused form; 1/2 around the Gram kernel)
        if (q0 == 0) DFS_CK(mark(6));
        if (fused_now) {
            DFS_CK(mark(7));
            DFS_CK(mark(1));
        }
        int sv_parts = p.pp.sv_grid;
        if (fused_now)
            DFS_CK(launch_gram_fused(p.tc, kq, S, p.n, m, lds, Vg, ldv, kg, Rpart, Sp, at<void>(h, p.off_P),
                                     at<int>(h, p.off_Rdy), h->dstat, h->num_sms, stream, &sv_parts));
        else
            DFS_CK(launch_sv_pack(p.pp, s_dtype, kq, q0 == 0 ? p.pack : 0, S, ni, m, lds, Vg, ldv, kg, Rpart, Sp,
                                  h->dstat, stream, rs ? rs + p.n_pad : nullptr, &sv_parts));
        if (fused_now) DFS_CK(mark(2));
        else if (q0 == 0) DFS_CK(mark(7));
        if (!p.ns)
            DFS_CK(launch_pass_reduce(p.f64, Rpart, sv_parts, ni, npi, kq, kg, nullptr, kq, lambda, R, kq, Z,
                                      nullptr, nullptr, h->dstat, 0, stream));
        if (center)  // b = P (O v) / sqrt(n)
            DFS_CK(launch_center_vec(p.f64, 0, ni, npi, kq, kg, R, nullptr, 0.0, Z, nullptr, h->dstat, 0, stream));
        if (q0 == 0) {
            // Algorithm 1 steps 1-2: W = S S^T + lambda I~ and its Cholesky factor
            void* P = at<void>(h, p.off_P);
            if (!p.fused) {
                DFS_CK(mark(1));
                if (p.tensor)
                    DFS_CK(launch_gram_tc(p.tc, p.s_dtype, S, p.n, p.m, lds, Sp, P, h->dstat, stream));
                else
                    DFS_CK(launch_gram_simt(p.s_dtype, p.f64, S, p.n, p.m, lds, p.nsplit, p.chunk, P, stream));
                DFS_CK(mark(2));
            }
            const double lam_g = center ? 0.0 : lambda;  // centring adds lambda after P G P / n
            if (p.tensor)
                DFS_CK(launch_gram_tc_finalize(p.tc, P, p.n, p.n_pad, lam_g, W, p.n_pad, stream, rs));
            else
                DFS_CK(launch_gram_finalize(p.f64, p.f64, gram_simt_tile(p.f64), P, p.nsplit, p.n, p.n_pad, lam_g,
                                            W, p.n_pad, stream));
            if (center) DFS_CK(launch_center_gram(p.f64, W, p.n_pad, ni, at<double>(h, p.off_Cg), lambda, stream));
            DFS_CK(mark(10));
            DFS_CK(launch_cholesky(p.f64, W, p.n_pad, p.n_pad, Linv, at<int>(h, p.off_Cf), h->dstat, stream,
                                   fp64_panel, h->chol_share));
            DFS_CK(mark(3));
        }
        // y0 = W^{-1} b by the two triangular solves (with the reduction of b = S v folded in)
        if (p.ns) {
            DFS_CK(launch_nspace(p.f64, kq, W, p.n_pad, npi, Linv, NS_MODE_REDUCE | NS_MODE_FWD | NS_MODE_BWD, Rpart,
                                 sv_parts, ni, kg, nullptr, lambda, nullptr, 0, R, Z, kq, nullptr, nullptr,
                                 h->smem_optin, h->dstat, 0, stream));
        } else {
            DFS_CK(launch_trsv(p.f64, 0, W, p.n_pad, npi, Linv, Z, kq, kg, kq, h->dstat, 0, stream));
            DFS_CK(launch_trsv(p.f64, 1, W, p.n_pad, npi, Linv, Z, kq, kg, kq, h->dstat, 0, stream));
        }
        DFS_CK(launch_refine_init(p.f64, Z, npi, kq, Y, R, bn2, h->dstat, stream));
        if (q0 == 0) DFS_CK(mark(4));
        const bool mark_pass = (q0 == 0);
        if (!p.tensor) {
            // x = (v - S^T y) / lambda
            if (center) DFS_CK(launch_center_vec(p.f64, 1, ni, npi, kq, kg, nullptr, Y, 0.0, nullptr, Yc, h->dstat, 0, stream));
            if (mark_pass) DFS_CK(mark(8));
            DFS_CK(launch_pass(p.pp, s_dtype, kq, S, ni, m, lds, Vg, ldv, kg, Yp, kq, lambda, Xg, ldx, nullptr,
                               U2part, 0, h->dstat, 0, stream));
            if (mark_pass) DFS_CK(mark(9));
        } else {
            // Steps 2 and 3 first read the packed BF16 tiles instead of S when they exist:
            // x_j = x_{j-1} - S_bf16^T dy_{j-1} / lambda (the tiles' rounding costs 2^-9 of a
            // correction of relative size delta_j, which the check adds to its estimate).  If that
            // does not converge, the full pass of step j recomputes x_j exactly and refinement goes
            // on; a step-3 correction then usually ends it (its delta_3 is a small multiple of
            // delta_2) one full pass earlier.  The last allowed step is always a full pass, so the
            // iteration budget is still decided on exact x.
            const bool fast = p.pack == 1 && !center && max_iter >= 3 && !p.f64 && kq <= 8 &&
                              tile_correct_fits((int)round_up(n, 256), kq, h->smem_optin);
            for (int it = 1; it <= max_iter; ++it) {
                const bool corrected = fast && (it == 2 || it == 3) && it < max_iter;
                if (corrected) {
                    if (mark_pass && it == 2) DFS_CK(mark(11));
                    int cparts = 0;
                    DFS_CK(launch_tile_correct(kq, Sp, ni, (int)round_up(n, 256), m, pack_kblocks(s_dtype, 1, m),
                                               static_cast<const float*>(Z), kg, lambda, static_cast<float*>(Xg), ldx,
                                               U2part, h->dstat, h->num_sms, stream, &cparts));
                    if (mark_pass && it == 2) DFS_CK(mark(12));
                    DFS_CK(launch_refine_check(U2part, cparts, U2, kq, kg, lambda, tol, it, max_iter, 1, h->dstat,
                                               stream));
                }
                if (center)
                    DFS_CK(launch_center_vec(p.f64, 1, ni, npi, kq, kg, nullptr, Y, 0.0, nullptr, Yc, h->dstat, 1, stream));
                // x_0 = v / lambda for the first pass; afterwards x_{j-1} is read from X itself (no
                // measurement after a correction: its check already took delta_2)
                if (mark_pass && it == 1) DFS_CK(mark(8));
                DFS_CK(launch_pass(p.pp, s_dtype, kq, S, ni, m, lds, Vg, ldv, kg, Yp, kq, lambda, Xg, ldx, Rpart,
                                   U2part, corrected ? 0 : (it == 1 ? 2 : 1), h->dstat, 1, stream));
                if (mark_pass && it == 1) DFS_CK(mark(9));
                if (!corrected)
                    DFS_CK(launch_refine_check(U2part, p.pp.uparts, U2, kq, kg, lambda, tol, it, max_iter, 0,
                                               h->dstat, stream));
                if (p.ns) {
                    DFS_CK(launch_nspace(p.f64, kq, W, p.n_pad, npi, Linv,
                                         NS_MODE_REDUCE | NS_MODE_LAMBDA_Y | NS_MODE_FWD | NS_MODE_BWD, Rpart,
                                         p.pp.nparts, ni, kg, Y, lambda, nullptr, 0, R, Z, kq, nullptr, nullptr,
                                         h->smem_optin, h->dstat, 1, stream));
                } else {
                    // r = S u - lambda y; centred: P (O u) / sqrt(n) - lambda y
                    DFS_CK(launch_pass_reduce(p.f64, Rpart, p.pp.nparts, ni, npi, kq, kg, center ? nullptr : Y, kq,
                                              lambda, R, kq, Z, nullptr, nullptr, h->dstat, 1, stream));
                    if (center)
                        DFS_CK(launch_center_vec(p.f64, 0, ni, npi, kq, kg, R, Y, lambda, Z, nullptr, h->dstat, 1,
                                                 stream));
                    DFS_CK(launch_trsv(p.f64, 0, W, p.n_pad, npi, Linv, Z, kq, kg, kq, h->dstat, 1, stream));
                    DFS_CK(launch_trsv(p.f64, 1, W, p.n_pad, npi, Linv, Z, kq, kg, kq, h->dstat, 1, stream));
                }
                DFS_CK(launch_refine_update(p.f64, Z, R, npi, kq, kg, Y, bn2, h->dstat, stream));
            }
            if (max_iter == 0) {
                if (center)
                    DFS_CK(launch_center_vec(p.f64, 1, ni, npi, kq, kg, nullptr, Y, 0.0, nullptr, Yc, h->dstat, 0, stream));
                if (mark_pass) DFS_CK(mark(8));
                DFS_CK(launch_pass(p.pp, s_dtype, kq, S, ni, m, lds, Vg, ldv, kg, Yp, kq, lambda, Xg, ldx, nullptr,
                                   U2part, 0, h->dstat, 0, stream));
                if (mark_pass) DFS_CK(mark(9));
            }
        }
    }
    DFS_CK(mark(5));
    h->timed = timed;
    if (timed) {
        h->tslot = slot;
        if (h->tpending < dfs_handle_s::kTimingSlots) ++h->tpending;
    }
    if (info) return fill_info(h, stream, info);
    return DFS_OK;
}

dfs_status grow(dfs_handle h, int i, size_t bytes) {
    if (bytes <= h->hbuf_bytes[i]) return DFS_OK;
    if (h->hbuf[i]) cudaFree(h->hbuf[i]);
    h->hbuf[i] = nullptr;
    h->hbuf_bytes[i] = 0;
    if (cudaMalloc(&h->hbuf[i], bytes) != cudaSuccess) {
        cudaGetLastError();
        return fail(h, DFS_ERR_NO_MEMORY, "cudaMalloc(%zu) for host-path staging failed", bytes);
    }
    h->hbuf_bytes[i] = bytes;
    return DFS_OK;
}

// Complex S = A + iB (Section 4, complex SR) natively on Z = [A; B] (2n x m, row stride lds; Zs
// is its first row), by the real kernels with the glue of complex.cu: the S v pass and the
// refinement passes read Z with two real right-hand sides per complex one, the Gram is Z Z^T, and
// the n-space steps solve the real 2n system R(W).  V and X are staged per group of kc complex
// right-hand sides as 2 kc real rows (the real parts, then the imaginary parts).
dfs_status solve_complex_device(dfs_handle h, const void* Zs, int s_dtype, int64_t n, int64_t m, int64_t lds,
                                const void* V_re, const void* V_im, int64_t k, int64_t ldv, double lambda, void* X_re,
                                void* X_im, int64_t ldx, const dfs_options* opt, cudaStream_t stream) {
    dfs_status s;
    int prec;
    if ((s = resolve_precision(h, s_dtype, opt ? opt->precision : DFS_PREC_AUTO, &prec)) != DFS_OK) return s;
    const int max_iter = (opt && opt->max_iter >= 0) ? opt->max_iter : 8;
    const double tol = (opt && opt->tol > 0.0) ? opt->tol : 1e-7;
    const int64_t n2 = 2 * n;
    // two pass columns per complex right-hand side, at most 8 (4 complex) per group
    const int kc_want = (int)(k < 4 ? k : 4);
    Plan p;
    const bool allow_fused = !(opt && (opt->flags & DFS_FLAG_TWO_KERNEL_GRAM));
    if ((s = make_plan(h, s_dtype, prec, n2, m, 2 * kc_want, &p, allow_fused)) != DFS_OK) return s;
    const int KQP = p.kq;
    const int kc = KQP / 2 < kc_want ? KQP / 2 : kc_want;
    if (kc < 1)
        return fail(h, DFS_ERR_UNSUPPORTED, "2n=%lld: the passes take fewer than two right-hand sides", (long long)n2);
    const int KQN = pow2_at_least(kc);
    // beyond the real plan: R(W) and the folded stopping sums
    const size_t es = p.f64 ? 8 : 4;
    const size_t np = (size_t)p.n_pad;
    const size_t off_Wc = align_up(p.total);
    const size_t off_U2c = align_up(off_Wc + np * np * es);
    const size_t off_dy = align_up(off_U2c + (size_t)std::max(p.pgrid, tile_correct_parts(h->num_sms)) * 2 * KQP * 8);
    const int n_rows_t = (int)round_up(n2, 256);  // rows of the packed tiles
    const size_t total = align_up(off_dy + (size_t)n_rows_t * KQP * sizeof(float));
    if ((s = ensure_ws(h, total, stream)) != DFS_OK) return s;
    const size_t vs = s_dtype == DFS_F64 ? 8 : 4;
    const int64_t ldc = round_up(m, 4);
    if ((s = grow(h, 1, (size_t)2 * k * ldc * vs)) != DFS_OK) return s;
    if ((s = grow(h, 2, (size_t)2 * kc * ldc * vs)) != DFS_OK) return s;
    char* Vall = static_cast<char*>(h->hbuf[1]);  // every group's rows, staged before X is written
    char* Xp = static_cast<char*>(h->hbuf[2]);
    h->last_precision = prec;
    h->timed = false;
    void* G = at<void>(h, p.off_W);
    void* Wc = at<void>(h, off_Wc);
    void* Linv = at<void>(h, p.off_Linv);
    double* Rpart = at<double>(h, p.off_Rpart);
    double* U2part = at<double>(h, p.off_U2part);
    double* U2c = at<double>(h, off_U2c);
    float* dy = at<float>(h, off_dy);  // the packed-tile correction's dy columns
    double* R = at<double>(h, p.off_R);
    void* Zv = at<void>(h, p.off_Z);
    double* Y = at<double>(h, p.off_Y);
    double* Yp = at<double>(h, p.off_Yc);  // the pass's y columns (2n x KQP)
    double* U2 = at<double>(h, p.off_U2);
    double* bn2 = at<double>(h, p.off_bn2);
    void* Sp = p.pack ? at<void>(h, p.off_Sp) : nullptr;
    float* rs = p.pack == 4 ? at<float>(h, p.off_Rs) : nullptr;
    const int n2i = (int)n2, npi = (int)p.n_pad, ni = (int)n;
    const int fp64_panel = opt && (opt->flags & DFS_FLAG_FP64_PANEL);
    const cudaMemcpyKind d2d = cudaMemcpyDeviceToDevice;

    // V staged per group: rows Re v_c0.., then Im v_c0.. (2 kg rows at row 2 c0)
    for (int64_t c0 = 0; c0 < k; c0 += kc) {
        const int kg = (int)(k - c0 < kc ? k - c0 : kc);
        char* Vg = Vall + 2 * c0 * ldc * vs;
        DFS_CK(cudaMemcpy2DAsync(Vg, ldc * vs, static_cast<const char*>(V_re) + c0 * ldv * vs, ldv * vs, m * vs, kg,
                                 d2d, stream));
        DFS_CK(cudaMemcpy2DAsync(Vg + kg * ldc * vs, ldc * vs, static_cast<const char*>(V_im) + c0 * ldv * vs,
                                 ldv * vs, m * vs, kg, d2d, stream));
    }
    DFS_CK(launch_status_reset(h->dstat, stream, h->test_wait_ns, h->test_fault));
    if (rs) DFS_CK(launch_row_scale(s_dtype, Zs, n2i, npi, m, lds, rs, h->dstat, stream));
    for (int64_t c0 = 0; c0 < k; c0 += kc) {
        const int kg = (int)(k - c0 < kc ? k - c0 : kc);  // complex right-hand sides of this group
        const char* Vp = Vall + 2 * c0 * ldc * vs;
        DFS_CK(launch_group_reset(h->dstat, stream));
        // b = S v from the S v pass over Z (the first group also writes Z's tensor-core tiles, and in
        // the fused form computes the Gram partials in the same kernel)
        int sv_parts = p.pp.sv_grid;
        const bool fused_now = c0 == 0 && p.fused;
        if (fused_now)
            DFS_CK(launch_gram_fused(p.tc, KQP, Zs, n2, m, lds, Vp, ldc, 2 * kg, Rpart, Sp, at<void>(h, p.off_P),
                                     at<int>(h, p.off_Rdy), h->dstat, h->num_sms, stream, &sv_parts));
        else
            DFS_CK(launch_sv_pack(p.pp, s_dtype, KQP, c0 == 0 ? p.pack : 0, Zs, n2i, m, lds, Vp, ldc, 2 * kg, Rpart,
                                  Sp, h->dstat, stream, rs ? rs + p.n_pad : nullptr, &sv_parts));
        DFS_CK(launch_complex_combine(p.f64, Rpart, sv_parts, ni, kg, KQP, nullptr, lambda, R, Zv, KQN, npi, nullptr, 0,
                                      nullptr, h->dstat, 0, stream));
        if (c0 == 0) {
            // W = S S^dagger + lambda I~ as R(W) from G = Z Z^T, and its Cholesky factor
            void* P = at<void>(h, p.off_P);
            if (p.tensor) {
                if (!p.fused) DFS_CK(launch_gram_tc(p.tc, s_dtype, Zs, n2, m, lds, Sp, P, h->dstat, stream));
                DFS_CK(launch_gram_tc_finalize(p.tc, P, n2, p.n_pad, 0.0, G, p.n_pad, stream, rs));
            } else {
                DFS_CK(launch_gram_simt(s_dtype, p.f64, Zs, n2, m, lds, p.nsplit, p.chunk, P, stream));
                DFS_CK(launch_gram_finalize(p.f64, p.f64, gram_simt_tile(p.f64), P, p.nsplit, n2, p.n_pad, 0.0, G,
                                            p.n_pad, stream));
            }
            DFS_CK(launch_complex_assemble(p.f64, G, p.n_pad, ni, npi, lambda, Wc, stream));
            DFS_CK(launch_cholesky(p.f64, Wc, p.n_pad, p.n_pad, Linv, at<int>(h, p.off_Cf), h->dstat, stream,
                                   fp64_panel, h->chol_share));
        }
        // z = R(W)^{-1} (the combined right-hand side in Zv), in place
        auto nspace_solve = [&](int honor) -> dfs_status {
            if (p.ns) {
                DFS_CK(launch_nspace(p.f64, KQN, Wc, p.n_pad, npi, Linv, NS_MODE_FWD | NS_MODE_BWD, nullptr, 0, n2i,
                                     kg, nullptr, lambda, Zv, KQN, nullptr, Zv, KQN, nullptr, nullptr, h->smem_optin,
                                     h->dstat, honor, stream));
            } else {
                DFS_CK(launch_trsv(p.f64, 0, Wc, p.n_pad, npi, Linv, Zv, KQN, kg, KQN, h->dstat, honor, stream));
                DFS_CK(launch_trsv(p.f64, 1, Wc, p.n_pad, npi, Linv, Zv, KQN, kg, KQN, h->dstat, honor, stream));
            }
            return DFS_OK;
        };
        if ((s = nspace_solve(0)) != DFS_OK) return s;
        DFS_CK(launch_refine_init(p.f64, Zv, npi, KQN, Y, R, bn2, h->dstat, stream));
        if (!p.tensor || max_iter == 0) {
            // x = (v - S^dagger y) / lambda
            DFS_CK(launch_complex_yexp(Y, KQN, ni, kg, KQP, Yp, h->dstat, 0, stream));
            DFS_CK(launch_pass(p.pp, s_dtype, KQP, Zs, n2i, m, lds, Vp, ldc, 2 * kg, Yp, KQP, lambda, Xp, ldc, nullptr,
                               U2part, 0, h->dstat, 0, stream));
        } else {
            // as the real path: steps 2 and 3 first take x_j = x_{j-1} - S_bf16^dagger dy_{j-1} / lambda
            // from Z's packed BF16 tiles; if that does not converge, the full pass of step j recomputes x_j
            const bool fast = p.pack == 1 && max_iter >= 3 && !p.f64 && tile_correct_fits(n_rows_t, KQP, h->smem_optin);
            for (int it = 1; it <= max_iter; ++it) {
                const bool corrected = fast && (it == 2 || it == 3) && it < max_iter;
                if (corrected) {
                    DFS_CK(launch_complex_dyexp(static_cast<const float*>(Zv), KQN, ni, kg, KQP, dy, n_rows_t, h->dstat,
                                                1, stream));
                    int cparts = 0;
                    DFS_CK(launch_tile_correct(KQP, Sp, n2i, n_rows_t, m, pack_kblocks(s_dtype, 1, m), dy, 2 * kg,
                                               lambda, reinterpret_cast<float*>(Xp), ldc, U2part, h->dstat,
                                               h->num_sms, stream, &cparts));
                    DFS_CK(launch_complex_combine(p.f64, nullptr, 0, ni, kg, KQP, nullptr, lambda, nullptr, nullptr, KQN,
                                                  npi, U2part, cparts, U2c, h->dstat, 1, stream));
                    DFS_CK(launch_refine_check(U2c, cparts, U2, KQN, kg, lambda, tol, it, max_iter, 1, h->dstat,
                                               stream));
                }
                DFS_CK(launch_complex_yexp(Y, KQN, ni, kg, KQP, Yp, h->dstat, 1, stream));
                DFS_CK(launch_pass(p.pp, s_dtype, KQP, Zs, n2i, m, lds, Vp, ldc, 2 * kg, Yp, KQP, lambda, Xp, ldc,
                                   Rpart, U2part, corrected ? 0 : (it == 1 ? 2 : 1), h->dstat, 1, stream));
                DFS_CK(launch_complex_combine(p.f64, Rpart, p.pp.nparts, ni, kg, KQP, Y, lambda, R, Zv, KQN, npi,
                                              corrected ? nullptr : U2part, p.pp.uparts, U2c, h->dstat, 1, stream));
                if (!corrected)
                    DFS_CK(launch_refine_check(U2c, p.pp.uparts, U2, KQN, kg, lambda, tol, it, max_iter, 0, h->dstat,
                                               stream));
                if ((s = nspace_solve(1)) != DFS_OK) return s;
                DFS_CK(launch_refine_update(p.f64, Zv, R, npi, KQN, kg, Y, bn2, h->dstat, stream));
            }
        }
        DFS_CK(cudaMemcpy2DAsync(static_cast<char*>(X_re) + c0 * ldx * vs, ldx * vs, Xp, ldc * vs, m * vs, kg, d2d,
                                 stream));
        DFS_CK(cudaMemcpy2DAsync(static_cast<char*>(X_im) + c0 * ldx * vs, ldx * vs, Xp + kg * ldc * vs, ldc * vs,
                                 m * vs, kg, d2d, stream));
    }
    return DFS_OK;
}

}  // namespace

extern "C" {

const char* dfs_status_string(int status) {
    switch (status) {
        case DFS_OK: return "DFS_OK";
        case DFS_ERR_INVALID_ARG: return "DFS_ERR_INVALID_ARG";
        case DFS_ERR_NOT_SPD: return "DFS_ERR_NOT_SPD";
        case DFS_ERR_NOT_CONVERGED: return "DFS_ERR_NOT_CONVERGED";
        case DFS_ERR_NONFINITE: return "DFS_ERR_NONFINITE";
        case DFS_ERR_TIMEOUT: return "DFS_ERR_TIMEOUT";
        case DFS_ERR_NO_MEMORY: return "DFS_ERR_NO_MEMORY";
        case DFS_ERR_CUDA: return "DFS_ERR_CUDA";
        case DFS_ERR_UNSUPPORTED: return "DFS_ERR_UNSUPPORTED";
        case DFS_ERR_BOUNDS: return "DFS_ERR_BOUNDS";
        default: return "DFS_ERR_UNKNOWN";
    }
}

const char* dfs_last_error(dfs_handle h) { return h ? h->err.c_str() : ""; }

int64_t dfs_kernel_launches(void) { return (int64_t)launch_counter().load(); }

dfs_status dfs_create(dfs_handle* out, int device) {
    if (!out) return DFS_ERR_INVALID_ARG;
    *out = nullptr;
    int count = 0;
    const cudaError_t ce = cudaGetDeviceCount(&count);
    if (ce != cudaSuccess || device < 0 || device >= count) {
        cudaGetLastError();
        return fail(nullptr, DFS_ERR_CUDA, "no CUDA device %d (%d visible: %s)", device, ce == cudaSuccess ? count : 0,
                    cudaGetErrorString(ce));
    }
    cudaDeviceProp prop;
    if (cudaGetDeviceProperties(&prop, device) != cudaSuccess)
        return fail(nullptr, DFS_ERR_CUDA, "cudaGetDeviceProperties(%d) failed", device);
    if (prop.major != 10 || prop.minor != 3)  // built for sm_103a only
        return fail(nullptr, DFS_ERR_UNSUPPORTED, "device %d is sm_%d%d; this build runs on sm_103a only", device,
                    prop.major, prop.minor);
    if (cudaSetDevice(device) != cudaSuccess) return fail(nullptr, DFS_ERR_CUDA, "cudaSetDevice(%d) failed", device);
    dfs_handle h = new dfs_handle_s();
    h->device = device;
    h->num_sms = prop.multiProcessorCount;
    h->smem_optin = prop.sharedMemPerBlockOptin;
    if (cudaMalloc(&h->dstat, sizeof(DevStatus)) != cudaSuccess) {
        delete h;
        cudaGetLastError();
        return fail(nullptr, DFS_ERR_NO_MEMORY, "cudaMalloc for the device status word failed");
    }
    cudaMemset(h->dstat, 0, sizeof(DevStatus));
    *out = h;
    return DFS_OK;
}

dfs_status dfs_destroy(dfs_handle h) {
    if (!h) return DFS_ERR_INVALID_ARG;
    cudaSetDevice(h->device);
    if (h->ws) cudaFree(h->ws);
    if (h->dstat) cudaFree(h->dstat);
    for (int sl = 0; sl < dfs_handle_s::kTimingSlots; ++sl)
        for (int i = 0; i < dfs_handle_s::kMarks; ++i)
            if (h->ev[sl][i]) cudaEventDestroy(h->ev[sl][i]);
    for (int i = 0; i < 3; ++i)
        if (h->hbuf[i]) cudaFree(h->hbuf[i]);
    if (h->bstat) cudaFree(h->bstat);
    for (int l = 0; l < dfs_handle_s::kMaxLanes; ++l) {
        if (h->lane[l]) dfs_destroy(h->lane[l]);
        if (h->lane_stream[l]) cudaStreamDestroy(h->lane_stream[l]);
        if (h->lane_done[l]) cudaEventDestroy(h->lane_done[l]);
    }
    if (h->fork_ev) cudaEventDestroy(h->fork_ev);
    for (int sl = 0; sl < 2; ++sl) {
        for (int b = 0; b < 2; ++b)
            if (h->abuf[sl][b]) cudaFree(h->abuf[sl][b]);
        if (h->slot_free[sl]) cudaEventDestroy(h->slot_free[sl]);
        if (h->slot_copied[sl]) cudaEventDestroy(h->slot_copied[sl]);
    }
    if (h->axbuf) cudaFree(h->axbuf);
    if (h->copy_stream) cudaStreamDestroy(h->copy_stream);
    delete h;
    return DFS_OK;
}

dfs_status dfs_reserve(dfs_handle h, int64_t n_max, int64_t m_max, int64_t k_max, int precision) {
    if (!h) return DFS_ERR_INVALID_ARG;
    if (n_max < 1 || m_max < 1 || k_max < 1) return fail(h, DFS_ERR_INVALID_ARG, "sizes must be >= 1");
    cudaSetDevice(h->device);
    size_t need = 0;
    const int dtypes[3] = {DFS_F32, DFS_BF16, DFS_F64};
    for (int dt : dtypes) {
        int prec;
        if (resolve_precision(h, dt, precision, &prec) != DFS_OK) continue;
        Plan p;
        if (make_plan(h, dt, prec, n_max, m_max, (int)k_max, &p) != DFS_OK) continue;
        if (p.total > need) need = p.total;
    }
    h->err.clear();
    if (need == 0) return fail(h, DFS_ERR_INVALID_ARG, "no dtype supports precision %d at these sizes", precision);
    return ensure_ws(h, need, nullptr);
}

dfs_status dfs_solve(dfs_handle h, const void* S, int s_dtype, int64_t n, int64_t m, int64_t lds, const void* V,
                     int64_t k, int64_t ldv, double lambda, void* X, int64_t ldx, const dfs_options* opt,
                     void* stream, dfs_info* info) {
    if (!h) return DFS_ERR_INVALID_ARG;
    h->err.clear();
    cudaSetDevice(h->device);
    return solve_device(h, S, s_dtype, n, m, lds, V, k, ldv, lambda, X, ldx, opt, (cudaStream_t)stream, info);
}

dfs_status dfs_solve_host(dfs_handle h, const void* S, int s_dtype, int64_t n, int64_t m, int64_t lds,
                          const void* V, int64_t k, int64_t ldv, double lambda, void* X, int64_t ldx,
                          const dfs_options* opt, void* stream_, dfs_info* info) {
    if (!h) return DFS_ERR_INVALID_ARG;
    h->err.clear();
    cudaSetDevice(h->device);
    cudaStream_t stream = (cudaStream_t)stream_;
    dfs_status s;
    if ((s = check_s(h, S, s_dtype, n, m, lds)) != DFS_OK) return s;
    if (!V || !X || k < 1 || ldv < m || ldx < m) return fail(h, DFS_ERR_INVALID_ARG, "bad V/X arguments");
    const size_t es = elem_size(s_dtype);
    const size_t vs = s_dtype == DFS_F64 ? 8 : 4;
    const int64_t lds_d = lds, ldv_d = round_up(m, 4), ldx_d = ldv_d;
    if ((s = grow(h, 0, (size_t)n * lds_d * es)) != DFS_OK) return s;
    if ((s = grow(h, 1, (size_t)k * ldv_d * vs)) != DFS_OK) return s;
    if ((s = grow(h, 2, (size_t)k * ldx_d * vs)) != DFS_OK) return s;
    DFS_CK(cudaMemcpyAsync(h->hbuf[0], S, (size_t)n * lds * es, cudaMemcpyHostToDevice, stream));
    DFS_CK(cudaMemcpy2DAsync(h->hbuf[1], ldv_d * vs, V, ldv * vs, m * vs, k, cudaMemcpyHostToDevice, stream));
    s = solve_device(h, h->hbuf[0], s_dtype, n, m, lds_d, h->hbuf[1], k, ldv_d, lambda, h->hbuf[2], ldx_d, opt,
                     stream, nullptr);
    if (s != DFS_OK) return s;
    DFS_CK(cudaMemcpy2DAsync(X, ldx * vs, h->hbuf[2], ldx_d * vs, m * vs, k, cudaMemcpyDeviceToHost, stream));
    return fill_info(h, stream, info);
}

// Grow a staging buffer; a buffer still in use by queued work is only replaced after the device
// has finished that work (cudaFree synchronizes).
static dfs_status grow_staging(dfs_handle h, void** buf, size_t* have, size_t need) {
    if (need <= *have) return DFS_OK;
    if (*buf) cudaFree(*buf);
    *buf = nullptr;
    *have = 0;
    if (cudaMalloc(buf, need) != cudaSuccess) {
        cudaGetLastError();
        return fail(h, DFS_ERR_NO_MEMORY, "cudaMalloc(%zu) for host-path staging failed", need);
    }
    *have = need;
    return DFS_OK;
}

dfs_status dfs_solve_host_async(dfs_handle h, const void* S, int s_dtype, int64_t n, int64_t m, int64_t lds,
                                const void* V, int64_t k, int64_t ldv, double lambda, void* X, int64_t ldx,
                                const dfs_options* opt, void* stream_) {
    if (!h) return DFS_ERR_INVALID_ARG;
    h->err.clear();
    cudaSetDevice(h->device);
    cudaStream_t stream = (cudaStream_t)stream_;
    dfs_status s;
    if ((s = check_s(h, S, s_dtype, n, m, lds)) != DFS_OK) return s;
    if (!V || !X || k < 1 || ldv < m || ldx < m) return fail(h, DFS_ERR_INVALID_ARG, "bad V/X arguments");
    const size_t es = elem_size(s_dtype);
    const size_t vs = s_dtype == DFS_F64 ? 8 : 4;
    const int64_t ldv_d = round_up(m, 4);
    if (!h->copy_stream) DFS_CK(cudaStreamCreateWithFlags(&h->copy_stream, cudaStreamNonBlocking));
    const int sl = h->aslot;
    h->aslot ^= 1;
    if (!h->slot_free[sl]) DFS_CK(cudaEventCreateWithFlags(&h->slot_free[sl], cudaEventDisableTiming));
    if (!h->slot_copied[sl]) DFS_CK(cudaEventCreateWithFlags(&h->slot_copied[sl], cudaEventDisableTiming));
    if ((s = grow_staging(h, &h->abuf[sl][0], &h->abuf_bytes[sl][0], (size_t)n * lds * es)) != DFS_OK) return s;
    if ((s = grow_staging(h, &h->abuf[sl][1], &h->abuf_bytes[sl][1], (size_t)k * ldv_d * vs)) != DFS_OK) return s;
    if ((s = grow_staging(h, &h->axbuf, &h->axbuf_bytes, (size_t)k * ldv_d * vs)) != DFS_OK) return s;
    // upload into this slot once the solve that last read it has finished
    if (h->slot_used[sl]) DFS_CK(cudaStreamWaitEvent(h->copy_stream, h->slot_free[sl], 0));
    DFS_CK(cudaMemcpyAsync(h->abuf[sl][0], S, (size_t)n * lds * es, cudaMemcpyHostToDevice, h->copy_stream));
    DFS_CK(cudaMemcpy2DAsync(h->abuf[sl][1], ldv_d * vs, V, ldv * vs, m * vs, k, cudaMemcpyHostToDevice,
                             h->copy_stream));
    DFS_CK(cudaEventRecord(h->slot_copied[sl], h->copy_stream));
    DFS_CK(cudaStreamWaitEvent(stream, h->slot_copied[sl], 0));
    s = solve_device(h, h->abuf[sl][0], s_dtype, n, m, lds, h->abuf[sl][1], k, ldv_d, lambda, h->axbuf, ldv_d, opt,
                     stream, nullptr);
    if (s != DFS_OK) return s;
    DFS_CK(cudaEventRecord(h->slot_free[sl], stream));
    h->slot_used[sl] = true;
    DFS_CK(cudaMemcpy2DAsync(X, ldx * vs, h->axbuf, ldv_d * vs, m * vs, k, cudaMemcpyDeviceToHost, stream));
    return DFS_OK;
}

dfs_status dfs_solve_complex(dfs_handle h, const void* S_re, const void* S_im, int s_dtype, int64_t n, int64_t m,
                             int64_t lds, const void* V_re, const void* V_im, int64_t k, int64_t ldv, double lambda,
                             void* X_re, void* X_im, int64_t ldx, const dfs_options* opt, void* stream_,
                             dfs_info* info) {
    if (!h) return DFS_ERR_INVALID_ARG;
    h->err.clear();
    cudaSetDevice(h->device);
    cudaStream_t stream = (cudaStream_t)stream_;
    dfs_status s;
    if ((s = check_s(h, S_re, s_dtype, n, m, lds)) != DFS_OK) return s;
    if ((s = check_s(h, S_im, s_dtype, n, m, lds)) != DFS_OK) return s;
    if ((s = check_lambda(h, lambda)) != DFS_OK) return s;
    if (!V_re || !V_im || !X_re || !X_im || k < 1 || ldv < m || ldx < m)
        return fail(h, DFS_ERR_INVALID_ARG, "bad V/X arguments");
    if (2 * n > 65536) return fail(h, DFS_ERR_UNSUPPORTED, "2n=%lld above the supported maximum 65536", (long long)(2 * n));
    if (opt && (opt->flags & DFS_FLAG_CENTER))
        return fail(h, DFS_ERR_UNSUPPORTED, "centring is not available for complex scores");
    // Z = [Re S; Im S]: the planes themselves when Im S follows Re S in one allocation (row n of
    // a 2n-row array), else a stacked copy
    const size_t es = elem_size(s_dtype);
    const void* Zs = S_re;
    if (static_cast<const char*>(S_im) != static_cast<const char*>(S_re) + (size_t)n * lds * es) {
        if ((s = grow(h, 0, (size_t)(2 * n) * lds * es)) != DFS_OK) return s;
        char* z = static_cast<char*>(h->hbuf[0]);
        DFS_CK(cudaMemcpy2DAsync(z, lds * es, S_re, lds * es, m * es, n, cudaMemcpyDeviceToDevice, stream));
        DFS_CK(cudaMemcpy2DAsync(z + (size_t)n * lds * es, lds * es, S_im, lds * es, m * es, n,
                                 cudaMemcpyDeviceToDevice, stream));
        Zs = z;
    }
    s = solve_complex_device(h, Zs, s_dtype, n, m, lds, V_re, V_im, k, ldv, lambda, X_re, X_im, ldx, opt, stream);
    if (s != DFS_OK) return s;
    return fill_info(h, stream, info);
}

dfs_status dfs_step_times(dfs_handle h, float* mean_ms, int* count) {
    if (!h || !mean_ms) return DFS_ERR_INVALID_ARG;
    cudaSetDevice(h->device);
    const int nsl = h->tpending;
    for (int i = 0; i < DFS_STEP_TIMES; ++i) mean_ms[i] = 0.0f;
    if (count) *count = nsl;
    if (nsl == 0) return DFS_OK;
    DFS_CK(cudaEventSynchronize(h->ev[h->tslot][5]));
    double acc[DFS_STEP_TIMES] = {};
    for (int j = 0; j < nsl; ++j) {
        const int sl = (h->tslot - j + dfs_handle_s::kTimingSlots) % dfs_handle_s::kTimingSlots;
        float ms[DFS_STEP_TIMES];
        step_ms(h->ev[sl], ms);
        for (int i = 0; i < DFS_STEP_TIMES; ++i) acc[i] += ms[i];
    }
    for (int i = 0; i < DFS_STEP_TIMES; ++i) mean_ms[i] = (float)(acc[i] / nsl);
    h->tpending = 0;
    return DFS_OK;
}

dfs_status dfs_set_test_fault(dfs_handle h, int fault, int64_t wait_limit_ns) {
    if (!h) return DFS_ERR_INVALID_ARG;
    if (fault < DFS_TEST_FAULT_NONE || fault > DFS_TEST_FAULT_FUSED_GRAM)
        return fail(h, DFS_ERR_INVALID_ARG, "unknown test fault %d", fault);
    h->test_fault = fault;
    h->test_wait_ns = wait_limit_ns > 0 ? (unsigned long long)wait_limit_ns : 0ull;
    return DFS_OK;
}

dfs_status dfs_sync_info(dfs_handle h, void* stream, dfs_info* info) {
    if (!h) return DFS_ERR_INVALID_ARG;
    cudaSetDevice(h->device);
    return fill_info(h, (cudaStream_t)stream, info);
}

dfs_status dfs_gram(dfs_handle h, const void* S, int s_dtype, int64_t n, int64_t m, int64_t lds, double lambda,
                    int precision, void* W, int64_t ldw, void* stream_) {
    if (!h) return DFS_ERR_INVALID_ARG;
    h->err.clear();
    cudaSetDevice(h->device);
    cudaStream_t stream = (cudaStream_t)stream_;
    dfs_status s;
    if ((s = check_s(h, S, s_dtype, n, m, lds)) != DFS_OK) return s;
    if ((s = check_lambda(h, lambda)) != DFS_OK) return s;
    if (!W || ldw < n) return fail(h, DFS_ERR_INVALID_ARG, "W is NULL or ldw < n");
    int prec;
    if ((s = resolve_precision(h, s_dtype, precision, &prec)) != DFS_OK) return s;
    Plan p;
    if ((s = make_plan(h, s_dtype, prec, n, m, 1, &p)) != DFS_OK) return s;
    if ((s = ensure_ws(h, p.total, stream)) != DFS_OK) return s;
    DFS_CK(launch_status_reset(h->dstat, stream, h->test_wait_ns, h->test_fault));
    return run_gram(h, p, S, lds, lambda, W, ldw, n, stream);
}

dfs_status dfs_cholesky(dfs_handle h, void* W, int w_dtype, int64_t n, int64_t ldw, void* stream_,
                        int64_t* failed_pivot) {
    if (!h) return DFS_ERR_INVALID_ARG;
    h->err.clear();
    cudaSetDevice(h->device);
    cudaStream_t stream = (cudaStream_t)stream_;
    if (failed_pivot) *failed_pivot = -1;
    if (!W || n < 1 || ldw < n || (w_dtype != DFS_F32 && w_dtype != DFS_F64))
        return fail(h, DFS_ERR_INVALID_ARG, "bad W arguments");
    const int f64 = w_dtype == DFS_F64;
    const int64_t n_pad = round_up(n, 128);
    const size_t es = f64 ? 8 : 4;
    dfs_status s;
    const size_t oI = align_up((size_t)n_pad * n_pad * es), oF = oI + align_up((size_t)n_pad * 32 * es);
    if ((s = ensure_ws(h, oF + cholesky_flag_bytes(n_pad), stream)) != DFS_OK) return s;
    void* Wp = h->ws;
    void* Linv = static_cast<char*>(h->ws) + oI;
    int* flags = reinterpret_cast<int*>(static_cast<char*>(h->ws) + oF);
    DFS_CK(launch_status_reset(h->dstat, stream, h->test_wait_ns, h->test_fault));
    DFS_CK(launch_pad_copy_in(f64, W, ldw, n, Wp, n_pad, stream));
    // the factorisation dfs_solve runs: FP32 W with FP32 diagonal blocks, FP64 W in FP64
    DFS_CK(launch_cholesky(f64, Wp, n_pad, n_pad, Linv, flags, h->dstat, stream, f64));
    DFS_CK(launch_copy_lower_out(f64, Wp, n_pad, W, ldw, n, stream));
    dfs_info info;
    s = fill_info(h, stream, &info);
    if (failed_pivot && info.failed_pivot >= 0) *failed_pivot = info.failed_pivot;
    return s;
}

dfs_status dfs_trsm(dfs_handle h, const void* L, int l_dtype, int64_t n, int64_t ldl, void* B, int64_t k,
                    int64_t ldb, int trans, void* stream_) {
    if (!h) return DFS_ERR_INVALID_ARG;
    h->err.clear();
    cudaSetDevice(h->device);
    cudaStream_t stream = (cudaStream_t)stream_;
    if (!L || !B || n < 1 || k < 1 || ldl < n || ldb < k || (l_dtype != DFS_F32 && l_dtype != DFS_F64) ||
        (trans != 0 && trans != 1))
        return fail(h, DFS_ERR_INVALID_ARG, "bad triangular-solve arguments");
    const int f64 = l_dtype == DFS_F64;
    const int64_t n_pad = round_up(n, 128);
    const size_t es = f64 ? 8 : 4;
    const int kmax = trsv_max_group((int)n_pad, (int)es, h->smem_optin);
    if (kmax < 1) return fail(h, DFS_ERR_UNSUPPORTED, "n too large for the on-chip triangular solve");
    int kq = pow2_at_least((int)(k < 8 ? k : 8));
    if (kq > kmax) kq = kmax;
    const size_t oL = 0, oI = align_up((size_t)n_pad * n_pad * es), oB = oI + align_up((size_t)n_pad * 32 * es);
    dfs_status s;
    if ((s = ensure_ws(h, oB + align_up((size_t)n_pad * kq * es), stream)) != DFS_OK) return s;
    void* Lp = static_cast<char*>(h->ws) + oL;
    void* Linv = static_cast<char*>(h->ws) + oI;
    void* Bp = static_cast<char*>(h->ws) + oB;
    DFS_CK(launch_status_reset(h->dstat, stream, h->test_wait_ns, h->test_fault));
    DFS_CK(launch_pad_copy_in(f64, L, ldl, n, Lp, n_pad, stream));
    DFS_CK(launch_diag_inverse(f64, Lp, n_pad, n_pad, Linv, h->dstat, stream));
    if (trans) DFS_CK(launch_mirror_lower(f64, Lp, n_pad, (int)n_pad, stream));
    for (int64_t q0 = 0; q0 < k; q0 += kq) {
        const int kg = (int)((k - q0) < kq ? (k - q0) : kq);
        void* Bg = static_cast<char*>(B) + q0 * es;
        DFS_CK(launch_copy_rhs_in(f64, Bg, ldb, n, kg, Bp, kq, n_pad, stream));
        if (nspace_slots((int)n_pad, kq, (int)es, h->smem_optin) >= 2)
            DFS_CK(launch_nspace(f64, kq, Lp, n_pad, (int)n_pad, Linv, trans ? NS_MODE_BWD : NS_MODE_FWD, nullptr, 0,
                                 (int)n, kg, nullptr, 0.0, Bp, kq, nullptr, Bp, kq, nullptr, nullptr, h->smem_optin,
                                 h->dstat, 0, stream));
        else
            DFS_CK(launch_trsv(f64, trans, Lp, n_pad, (int)n_pad, Linv, Bp, kq, kg, kq, h->dstat, 0, stream));
        DFS_CK(launch_copy_rhs_out(f64, Bp, kq, n, kg, Bg, ldb, stream));
    }
    return fill_info(h, stream, nullptr);
}

dfs_status dfs_fisher_pass(dfs_handle h, const void* S, int s_dtype, int64_t n, int64_t m, int64_t lds,
                           const void* V, int64_t k, int64_t ldv, const double* Y, int64_t ldy, double lambda,
                           void* X, int64_t ldx, double* R, int64_t ldr, void* stream_) {
    if (!h) return DFS_ERR_INVALID_ARG;
    h->err.clear();
    cudaSetDevice(h->device);
    cudaStream_t stream = (cudaStream_t)stream_;
    dfs_status s;
    if ((s = check_s(h, S, s_dtype, n, m, lds)) != DFS_OK) return s;
    if ((s = check_lambda(h, lambda)) != DFS_OK) return s;
    if (!V || k < 1 || ldv < m) return fail(h, DFS_ERR_INVALID_ARG, "bad V arguments");
    if (X && ldx < m) return fail(h, DFS_ERR_INVALID_ARG, "ldx < m");
    if (Y && ldy < k) return fail(h, DFS_ERR_INVALID_ARG, "ldy < k");
    if (R && ldr < k) return fail(h, DFS_ERR_INVALID_ARG, "ldr < k");
    int kq = pow2_at_least((int)k);
    const int kmax = pass_max_group((int)n, s_dtype, h->smem_optin);
    if (kmax < 1) return fail(h, DFS_ERR_UNSUPPORTED, "n too large for the pass kernel");
    if (kq > kmax) kq = kmax;
    const PassPlan pp = pass_make_plan((int)n, kq, s_dtype, h->num_sms, m, h->smem_optin, X != nullptr);
    const int grid = std::max(pass_partial_rows(pp), pp.uparts);
    const size_t oR = 0, oU = align_up((size_t)grid * n * kq * 8), oU2 = oU + align_up((size_t)grid * 2 * kq * 8);
    if ((s = ensure_ws(h, oU2 + 128, stream)) != DFS_OK) return s;
    double* Rpart = reinterpret_cast<double*>(static_cast<char*>(h->ws) + oR);
    double* U2part = reinterpret_cast<double*>(static_cast<char*>(h->ws) + oU);
    const size_t vs = s_dtype == DFS_F64 ? 8 : 4;
    DFS_CK(launch_status_reset(h->dstat, stream, h->test_wait_ns, h->test_fault));
    for (int64_t q0 = 0; q0 < k; q0 += kq) {
        const int kg = (int)((k - q0) < kq ? (k - q0) : kq);
        const void* Vg = static_cast<const char*>(V) + q0 * ldv * vs;
        void* Xg = X ? static_cast<char*>(X) + q0 * ldx * vs : nullptr;
        const double* Yg = Y ? Y + q0 : nullptr;
        DFS_CK(launch_pass(pp, s_dtype, kq, S, (int)n, m, lds, Vg, ldv, kg, Yg, Y ? ldy : kq, lambda, Xg, ldx,
                           R ? Rpart : nullptr, U2part, 0, h->dstat, 0, stream));
        if (R)
            DFS_CK(launch_pass_reduce(0, Rpart, pp.nparts, (int)n, (int)n, kq, kg, Yg, ldy, lambda, R + q0, ldr, nullptr,
                                      nullptr, nullptr, h->dstat, 0, stream));
    }
    return DFS_OK;
}

// ---- batches of independent problems ------------------------------------------------------

static dfs_status check_batch(dfs_handle h, const dfs_problem* problems, int count, int s_dtype) {
    if (!problems || count < 1) return fail(h, DFS_ERR_INVALID_ARG, "empty problem list");
    for (int i = 0; i < count; ++i) {
        const dfs_problem& q = problems[i];
        dfs_status s;
        if ((s = check_s(h, q.S, s_dtype, q.n, q.m, q.lds)) != DFS_OK) return s;
        if ((s = check_lambda(h, q.lambda)) != DFS_OK) return s;
        if (!q.V || !q.X || q.k < 1 || q.ldv < q.m || q.ldx < q.m)
            return fail(h, DFS_ERR_INVALID_ARG, "problem %d: bad V/X arguments", i);
    }
    return DFS_OK;
}

// Lanes: problems are dealt longest first (estimated cost n^2 m + 4 n m k: the Gram and the
// passes over S) to the lane with the least work so far; each lane solves its problems in order
// on its own stream and workspace.  With one lane this is a plain loop on the caller's stream.
// Eight lanes: 64 problems of n ~ U{64..1024}, m log-uniform in [1e4, 5e5] ran 1.63x faster than
// one stream with four lanes, 1.78x with eight, 1.80x with sixteen.  Returns the lane count;
// `order` receives the problems longest first, `lane_of` each problem's lane.
static int schedule_batch(dfs_handle h, const dfs_problem* problems, int count, std::vector<int>& order,
                          std::vector<int>& lane_of) {
    const int L = count < h->batch_lanes ? count : h->batch_lanes;
    order.resize(count);
    for (int i = 0; i < count; ++i) order[i] = i;
    auto cost = [&](int i) {
        const dfs_problem& q = problems[i];
        return (double)q.n * (double)q.n * (double)q.m + 4.0 * (double)q.n * (double)q.m * (double)q.k;
    };
    std::stable_sort(order.begin(), order.end(), [&](int a, int b) { return cost(a) > cost(b); });
    lane_of.assign(count, 0);
    std::vector<double> load(L, 0.0);
    for (int i : order) {
        int best = 0;
        for (int l = 1; l < L; ++l)
            if (load[l] < load[best]) best = l;
        lane_of[i] = best;
        load[best] += cost(i);
    }
    return L;
}

static bool capturing(cudaStream_t stream) {
    cudaStreamCaptureStatus cs = cudaStreamCaptureStatusNone;
    return cudaStreamIsCapturing(stream, &cs) == cudaSuccess && cs != cudaStreamCaptureStatusNone;
}

// The per-problem status array and, for L > 1, lanes 0..L-1 with their streams and events.
// Nothing is created while `stream` is being captured (that is an error).
static dfs_status prepare_batch(dfs_handle h, int count, int L, cudaStream_t stream) {
    const bool cap = capturing(stream);
    if (count > h->bstat_count) {
        if (cap) return fail(h, DFS_ERR_NO_MEMORY, "batch status array must grow during stream capture; call dfs_plan_batched first");
        if (h->bstat) cudaFree(h->bstat);
        h->bstat = nullptr;
        h->bstat_count = 0;
        if (cudaMalloc(&h->bstat, sizeof(int) * count) != cudaSuccess) {
            cudaGetLastError();
            return fail(h, DFS_ERR_NO_MEMORY, "cudaMalloc for batch status failed");
        }
        h->bstat_count = count;
    }
    if (L < 2) return DFS_OK;
    for (int l = 0; l < L; ++l) {
        if (!h->lane[l] || !h->lane_stream[l] || !h->lane_done[l]) {
            if (cap) return fail(h, DFS_ERR_NO_MEMORY, "batch lane %d must be created during stream capture; call dfs_plan_batched first", l);
            if (!h->lane[l]) {
                dfs_status s = dfs_create(&h->lane[l], h->device);
                if (s != DFS_OK) return fail(h, s, "creating batch lane %d failed", l);
            }
            if (!h->lane_stream[l]) DFS_CK(cudaStreamCreateWithFlags(&h->lane_stream[l], cudaStreamNonBlocking));
            if (!h->lane_done[l]) DFS_CK(cudaEventCreateWithFlags(&h->lane_done[l], cudaEventDisableTiming));
        }
        // every lane's cooperative Cholesky fits on the device at the same time as the others'
        h->lane[l]->chol_share = L;
        h->lane[l]->lane_handle = true;
        // the lane's other kernels size their grids for its share of the SMs, so that the small
        // problems' latency-bound kernels leave room for the other lanes'
        h->lane[l]->num_sms = h->num_sms / h->batch_share > 0 ? h->num_sms / h->batch_share : 1;
    }
    if (!h->fork_ev) {
        if (cap) return fail(h, DFS_ERR_NO_MEMORY, "batch fork event must be created during stream capture; call dfs_plan_batched first");
        DFS_CK(cudaEventCreateWithFlags(&h->fork_ev, cudaEventDisableTiming));
    }
    return DFS_OK;
}

dfs_status dfs_plan_batched(dfs_handle h, const dfs_problem* problems, int count, int s_dtype,
                            const dfs_options* opt, size_t* workspace_bytes) {
    if (workspace_bytes) *workspace_bytes = 0;
    if (!h) return DFS_ERR_INVALID_ARG;
    h->err.clear();
    cudaSetDevice(h->device);
    dfs_status s;
    if ((s = check_batch(h, problems, count, s_dtype)) != DFS_OK) return s;
    int prec;
    if ((s = resolve_precision(h, s_dtype, opt ? opt->precision : DFS_PREC_AUTO, &prec)) != DFS_OK) return s;
    std::vector<int> order, lane_of;
    const int L = schedule_batch(h, problems, count, order, lane_of);
    if ((s = prepare_batch(h, count, L, nullptr)) != DFS_OK) return s;
    // each lane's workspace: the largest plan among the problems dealt to it (planned on the lane,
    // with its share of the SMs and the caller's group size)
    const int kq_cap = opt ? (opt->flags >> 8) & 15 : 0;
    std::vector<size_t> need(L, 0);
    for (int i = 0; i < count; ++i) {
        const dfs_problem& q = problems[i];
        Plan p;
        if ((s = make_plan(L == 1 ? h : h->lane[lane_of[i]], s_dtype, prec, q.n, q.m, (int)q.k, &p, true, kq_cap)) !=
            DFS_OK)
            return s;
        if (p.total > need[lane_of[i]]) need[lane_of[i]] = p.total;
    }
    size_t held = sizeof(int) * (size_t)h->bstat_count;
    for (int l = 0; l < L; ++l) {
        dfs_handle lh = L == 1 ? h : h->lane[l];
        if ((s = ensure_ws(lh, need[l], nullptr)) != DFS_OK) return L == 1 ? s : fail(h, s, "lane %d: %s", l, lh->err.c_str());
        held += lh->ws_bytes;
    }
    if (workspace_bytes) *workspace_bytes = held;
    return DFS_OK;
}

dfs_status dfs_solve_batched(dfs_handle h, const dfs_problem* problems, int count, int s_dtype,
                             const dfs_options* opt, void* stream_, int* status_out) {
    if (!h) return DFS_ERR_INVALID_ARG;
    h->err.clear();
    cudaSetDevice(h->device);
    cudaStream_t stream = (cudaStream_t)stream_;
    dfs_status s;
    if ((s = check_batch(h, problems, count, s_dtype)) != DFS_OK) return s;
    std::vector<int> order, lane_of;
    const int L = schedule_batch(h, problems, count, order, lane_of);
    if ((s = prepare_batch(h, count, L, stream)) != DFS_OK) return s;
    h->bstat_used = count;
    if (L == 1) {
        for (int i : order) {
            const dfs_problem& q = problems[i];
            s = solve_device(h, q.S, s_dtype, q.n, q.m, q.lds, q.V, q.k, q.ldv, q.lambda, q.X, q.ldx, opt, stream,
                             nullptr);
            if (s != DFS_OK) return s;
            DFS_CK(launch_status_save(h->dstat, h->bstat + i, stream));
        }
    } else {
        DFS_CK(cudaEventRecord(h->fork_ev, stream));
        for (int l = 0; l < L; ++l) DFS_CK(cudaStreamWaitEvent(h->lane_stream[l], h->fork_ev, 0));
        for (int i : order) {
            const dfs_problem& q = problems[i];
            dfs_handle lh = h->lane[lane_of[i]];
            cudaStream_t ls = h->lane_stream[lane_of[i]];
            s = solve_device(lh, q.S, s_dtype, q.n, q.m, q.lds, q.V, q.k, q.ldv, q.lambda, q.X, q.ldx, opt, ls,
                             nullptr);
            if (s != DFS_OK) return fail(h, s, "problem %d: %s", i, lh->err.c_str());
            DFS_CK(launch_status_save(lh->dstat, h->bstat + i, ls));
        }
        for (int l = 0; l < L; ++l) {
            DFS_CK(cudaEventRecord(h->lane_done[l], h->lane_stream[l]));
            DFS_CK(cudaStreamWaitEvent(stream, h->lane_done[l], 0));
        }
    }
    if (status_out) return dfs_batched_status(h, status_out, count, stream_);
    return DFS_OK;
}

dfs_status dfs_set_batch_lanes(dfs_handle h, int lanes, int share) {
    if (!h) return DFS_ERR_INVALID_ARG;
    h->err.clear();
    if (lanes < 1 || lanes > dfs_handle_s::kMaxLanes || share < 1 || share > 16)
        return fail(h, DFS_ERR_INVALID_ARG, "batch lanes %d (1..%d) or share %d (1..16) out of range", lanes,
                    dfs_handle_s::kMaxLanes, share);
    h->batch_lanes = lanes;
    h->batch_share = share;
    return DFS_OK;
}

dfs_status dfs_get_batch_lanes(dfs_handle h, int* lanes, int* share) {
    if (!h) return DFS_ERR_INVALID_ARG;
    if (lanes) *lanes = h->batch_lanes;
    if (share) *share = h->batch_share;
    return DFS_OK;
}

// ---- autotuner of the batched path -----------------------------------------------------------
// The batch's key: its size, dtype, precision and a hash of its problems' shapes (n, m, k), sorted
// so that the order of the list does not matter.
static std::string batch_key(const dfs_problem* problems, int count, int s_dtype, int prec) {
    std::vector<std::array<int64_t, 3>> shapes(count);
    for (int i = 0; i < count; ++i) shapes[i] = {problems[i].n, problems[i].m, problems[i].k};
    std::sort(shapes.begin(), shapes.end());
    uint64_t hsh = 1469598103934665603ull;  // FNV-1a over the shape words
    for (const auto& sh : shapes)
        for (int64_t v : sh)
            for (int b = 0; b < 8; ++b) {
                hsh ^= (uint64_t)((v >> (8 * b)) & 0xff);
                hsh *= 1099511628211ull;
            }
    char buf[96];
    std::snprintf(buf, sizeof(buf), "c%d_d%d_p%d_%016llx", count, s_dtype, prec, (unsigned long long)hsh);
    return buf;
}

// Finds `"field": <int>` in a JSON line (a flat object this file writes itself).
static bool json_int(const std::string& line, const char* field, int* out) {
    const std::string tag = std::string("\"") + field + "\":";
    const size_t p = line.find(tag);
    return p != std::string::npos && std::sscanf(line.c_str() + p + tag.size(), " %d", out) == 1;
}
static bool json_str(const std::string& line, const char* field, std::string* out) {
    const std::string tag = std::string("\"") + field + "\": \"";
    const size_t p = line.find(tag);
    if (p == std::string::npos) return false;
    const size_t e = line.find('"', p + tag.size());
    if (e == std::string::npos) return false;
    *out = line.substr(p + tag.size(), e - p - tag.size());
    return true;
}

dfs_status dfs_autotune_batched(dfs_handle h, const dfs_problem* problems, int count, int s_dtype,
                                const dfs_options* opt, const char* cache_path, void* stream_, int* lanes_out,
                                int* share_out, float* ms_out) {
    if (!h) return DFS_ERR_INVALID_ARG;
    h->err.clear();
    cudaSetDevice(h->device);
    cudaStream_t stream = (cudaStream_t)stream_;
    dfs_status s;
    if ((s = check_batch(h, problems, count, s_dtype)) != DFS_OK) return s;
    if (capturing(stream)) return fail(h, DFS_ERR_INVALID_ARG, "dfs_autotune_batched cannot run under stream capture");
    int prec;
    if ((s = resolve_precision(h, s_dtype, opt ? opt->precision : DFS_PREC_AUTO, &prec)) != DFS_OK) return s;
    cudaDeviceProp prop;
    DFS_CK(cudaGetDeviceProperties(&prop, h->device));
    const std::string gpu = prop.name, key = batch_key(problems, count, s_dtype, prec);
    // a recorded choice for this GPU and batch (the last line for the key wins): use it untimed
    if (cache_path) {
        bool hit = false;
        if (FILE* fp = std::fopen(cache_path, "r")) {
            char line[512];
            while (std::fgets(line, sizeof(line), fp)) {
                const std::string ln = line;
                std::string g, b;
                int lanes = 0, share = 0;
                if (json_str(ln, "gpu", &g) && json_str(ln, "batch", &b) && g == gpu && b == key &&
                    json_int(ln, "lanes", &lanes) && json_int(ln, "share", &share) && lanes >= 1 &&
                    lanes <= dfs_handle_s::kMaxLanes && share >= 1 && share <= 16) {
                    h->batch_lanes = lanes;
                    h->batch_share = share;
                    hit = true;
                }
            }
            std::fclose(fp);
        }
        if (hit) {
            if (lanes_out) *lanes_out = h->batch_lanes;
            if (share_out) *share_out = h->batch_share;
            if (ms_out) *ms_out = 0.f;  // nothing was timed
            return DFS_OK;
        }
    }
    static const int cand[][2] = {{8, 1}, {8, 2}, {8, 4}, {8, 8}, {16, 4}, {16, 8}, {4, 1}, {4, 2}};
    cudaEvent_t e0, e1;
    DFS_CK(cudaEventCreate(&e0));
    DFS_CK(cudaEventCreate(&e1));
    float best = -1.f;
    int best_l = h->batch_lanes, best_s = h->batch_share;
    for (const auto& c : cand) {
        h->batch_lanes = c[0];
        h->batch_share = c[1];
        size_t held = 0;
        if ((s = dfs_plan_batched(h, problems, count, s_dtype, opt, &held)) != DFS_OK) break;
        if ((s = dfs_solve_batched(h, problems, count, s_dtype, opt, stream, nullptr)) != DFS_OK) break;  // warm-up
        DFS_CK(cudaEventRecord(e0, stream));
        for (int r = 0; r < 2 && s == DFS_OK; ++r) s = dfs_solve_batched(h, problems, count, s_dtype, opt, stream, nullptr);
        if (s != DFS_OK) break;
        DFS_CK(cudaEventRecord(e1, stream));
        DFS_CK(cudaEventSynchronize(e1));
        float ms = 0.f;
        DFS_CK(cudaEventElapsedTime(&ms, e0, e1));
        ms *= 0.5f;
        if (best < 0.f || ms < best) {
            best = ms;
            best_l = c[0];
            best_s = c[1];
        }
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    h->batch_lanes = best_l;
    h->batch_share = best_s;
    if (s != DFS_OK) return s;
    // the device status of the last timed run (every problem solved)
    std::vector<int> st(count);
    if ((s = dfs_batched_status(h, st.data(), count, stream_)) != DFS_OK && s != DFS_ERR_NOT_CONVERGED) return s;
    if (cache_path) {
        if (FILE* fp = std::fopen(cache_path, "a")) {
            std::fprintf(fp, "{\"gpu\": \"%s\", \"batch\": \"%s\", \"lanes\": %d, \"share\": %d, \"ms\": %.4f}\n",
                         gpu.c_str(), key.c_str(), best_l, best_s, best);
            std::fclose(fp);
        }
    }
    if (lanes_out) *lanes_out = best_l;
    if (share_out) *share_out = best_s;
    if (ms_out) *ms_out = best;
    return DFS_OK;
}

dfs_status dfs_batched_status(dfs_handle h, int* status_out, int count, void* stream_) {
    if (!h) return DFS_ERR_INVALID_ARG;
    h->err.clear();
    cudaSetDevice(h->device);
    if (!status_out || count < 0 || count > h->bstat_used)
        return fail(h, DFS_ERR_INVALID_ARG, "count %d is not within the last batch's %d problems", count, h->bstat_used);
    if (count == 0) return DFS_OK;
    cudaStream_t stream = (cudaStream_t)stream_;
    DFS_CK(cudaMemcpyAsync(status_out, h->bstat, sizeof(int) * count, cudaMemcpyDeviceToHost, stream));
    DFS_CK(cudaStreamSynchronize(stream));
    for (int i = 0; i < count; ++i)
        if (status_out[i] != DFS_OK)
            return fail(h, (dfs_status)status_out[i], "problem %d: %s", i, dfs_status_string(status_out[i]));
    return DFS_OK;
}

}  // extern "C"
