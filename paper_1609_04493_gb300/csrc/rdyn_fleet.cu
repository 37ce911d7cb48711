// rdyn_fleet.cu -- many chains of different lengths, mixed inverse / forward
// dynamics requests in one call (rd_fleet_*, rd_plan_*, fleet_batch).
// All allocation happens when fleets and plans are created.
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <atomic>
#include <new>
#include <numeric>
#include <type_traits>
#include <vector>

#include "fleet.cuh"
#include "rdyn_internal.h"

struct rd_fleet {
    int device = 0;
    int nrobots = 0;
    long long total_links = 0;
    std::vector<int> n;  // host copy
    float *c32 = nullptr;     // [links][16] common-normal constants
    double *c64 = nullptr;    // same in FP64
    double *aba64 = nullptr;  // [links][32] FP64 forward-dynamics records
    rdyn::DF *abadf = nullptr;  // the same split into double-float pairs (FP32 data)
    int *robot_n = nullptr, *robot_link = nullptr;
    float *gb32 = nullptr, *tn32 = nullptr;  // [robots][12] boundary frames
    double *gb64 = nullptr, *tn64 = nullptr;
};

struct rd_plan {
    const rd_fleet *fleet = nullptr;
    int dtype = RD_F32;
    int R = 0;
    long long total_joints = 0;
    std::vector<long long> off;               // user order
    std::vector<std::pair<int, int>> groups;  // sorted positions [begin, end) of equal (kind, n)
    int *order = nullptr, *req_robot = nullptr, *req_kind = nullptr, *counter = nullptr;
    long long *req_off = nullptr;
    long long *group_ws = nullptr, *group_wz = nullptr;  // per 32 sorted positions
    // leading groups of 32 sorted positions whose forward-dynamics requests
    // run the bias sweeps in double-float (FP32 plans; longest chain beyond
    // RD_ABA_EXTENDED_BIAS_LINKS)
    int ext_groups = 0;
    // per group of 32 sorted positions: the longest forward-dynamics chain that
    // starts it (0 when it starts with inverse dynamics), for the two-warp
    // schedule's threshold
    std::vector<int> group_fd_n;
    unsigned char *ws = nullptr;
    size_t ws_bytes = 0;
    int sms = 0;
    // side streams for RD_SCHED_PER_GROUP (fork / join through events)
    static constexpr int kSide = 8;
    cudaStream_t side[kSide] = {};
    cudaEvent_t fork = nullptr, join[kSide] = {};
};

namespace {

template <typename X>
cudaError_t upload(X **dst, const X *src, size_t count)
{
    cudaError_t e = cudaMalloc(dst, std::max<size_t>(count, 1) * sizeof(X));
    if (e == cudaSuccess && count) e = cudaMemcpy(*dst, src, count * sizeof(X), cudaMemcpyHostToDevice);
    return e;
}

}  // namespace

extern "C" void rd_fleet_destroy(rd_fleet *f)
{
    if (!f) return;
    cudaFree(f->c32);
    cudaFree(f->c64);
    cudaFree(f->aba64);
    cudaFree(f->abadf);
    cudaFree(f->robot_n);
    cudaFree(f->robot_link);
    cudaFree(f->gb32);
    cudaFree(f->gb64);
    cudaFree(f->tn32);
    cudaFree(f->tn64);
    delete f;
}

extern "C" int rd_fleet_create(int nrobots, const int *n, const double *M, const double *S,
                               const double *inertia, rd_fleet **out)
{
    g_rd_error.clear();
    if (!out) return rd_fail(RD_ERR_ARG, "rd_fleet_create: out is null");
    *out = nullptr;
    if (nrobots < 1) return rd_fail(RD_ERR_RANGE, "rd_fleet_create: nrobots = %d", nrobots);
    if (!n || !M || !S || !inertia) return rd_fail(RD_ERR_ARG, "rd_fleet_create: null array");
    std::vector<double> all64, allaba;
    std::vector<int> link(nrobots);
    std::vector<double> tn((size_t)nrobots * 12), gb((size_t)nrobots * 12);
    long long lo = 0;
    for (int r = 0; r < nrobots; ++r) {
        if (n[r] < 1 || n[r] > RD_MAX_LINKS)
            return rd_fail(RD_ERR_RANGE, "rd_fleet_create: robot %d has n = %d outside [1, %d]", r,
                           n[r], RD_MAX_LINKS);
        std::vector<double> c, dh, aba;
        double TnR[9], Tnp[3], GBR[9], GBp[3], phi = 0.0;
        int rc = rd_build_chain(n[r], M + 12 * lo, S + 6 * lo, inertia + 10 * lo, c, TnR, Tnp);
        if (rc == RD_OK) rc = rd_build_dh(n[r], c, dh, GBR, GBp, &phi);
        if (rc) {
            std::string msg = g_rd_error;
            return rd_fail(rc, "rd_fleet_create: robot %d: %s", r, msg.c_str());
        }
        rd_build_aba64(n[r], dh, aba);
        link[r] = (int)lo;
        all64.insert(all64.end(), dh.begin(), dh.end());
        allaba.insert(allaba.end(), aba.begin(), aba.end());
        // F_{n+1} goes from frame n to D_{n-1}: the joint frame of link n
        // turned by phi about its z axis, R' = R Rz(phi), same origin
        const double cp = std::cos(phi), sp = std::sin(phi);
        for (int i = 0; i < 3; ++i) {
            tn[(size_t)r * 12 + 3 * i + 0] = TnR[3 * i] * cp + TnR[3 * i + 1] * sp;
            tn[(size_t)r * 12 + 3 * i + 1] = -TnR[3 * i] * sp + TnR[3 * i + 1] * cp;
            tn[(size_t)r * 12 + 3 * i + 2] = TnR[3 * i + 2];
        }
        for (int k = 0; k < 3; ++k) tn[(size_t)r * 12 + 9 + k] = Tnp[k];
        for (int k = 0; k < 9; ++k) gb[(size_t)r * 12 + k] = GBR[k];
        for (int k = 0; k < 3; ++k) gb[(size_t)r * 12 + 9 + k] = GBp[k];
        lo += n[r];
    }
    rd_fleet *f = new (std::nothrow) rd_fleet();
    if (!f) return rd_fail(RD_ERR_ALLOC, "rd_fleet_create: host allocation failed");
    f->nrobots = nrobots;
    f->total_links = lo;
    f->n.assign(n, n + nrobots);
    cudaError_t e = cudaGetDevice(&f->device);
    std::vector<float> all32(all64.begin(), all64.end());
    std::vector<float> tn32(tn.begin(), tn.end()), gb32(gb.begin(), gb.end());
    if (e == cudaSuccess) e = upload(&f->c64, all64.data(), all64.size());
    if (e == cudaSuccess) e = upload(&f->c32, all32.data(), all32.size());
    std::vector<rdyn::DF> alldf(allaba.size());
    for (size_t k = 0; k < allaba.size(); ++k) alldf[k] = rdyn::df_split_host(allaba[k]);
    if (e == cudaSuccess) e = upload(&f->aba64, allaba.data(), allaba.size());
    if (e == cudaSuccess) e = upload(&f->abadf, alldf.data(), alldf.size());
    if (e == cudaSuccess) e = upload(&f->robot_n, n, (size_t)nrobots);
    if (e == cudaSuccess) e = upload(&f->robot_link, link.data(), link.size());
    if (e == cudaSuccess) e = upload(&f->tn64, tn.data(), tn.size());
    if (e == cudaSuccess) e = upload(&f->tn32, tn32.data(), tn32.size());
    if (e == cudaSuccess) e = upload(&f->gb64, gb.data(), gb.size());
    if (e == cudaSuccess) e = upload(&f->gb32, gb32.data(), gb32.size());
    if (e != cudaSuccess) {
        rd_fleet_destroy(f);
        return rd_fail(RD_ERR_ALLOC, "rd_fleet_create: %s", cudaGetErrorString(e));
    }
    *out = f;
    return RD_OK;
}

extern "C" void rd_plan_destroy(rd_plan *p)
{
    if (!p) return;
    cudaFree(p->order);
    cudaFree(p->req_robot);
    cudaFree(p->req_kind);
    cudaFree(p->counter);
    cudaFree(p->req_off);
    cudaFree(p->group_ws);
    cudaFree(p->group_wz);
    cudaFree(p->ws);
    for (int k = 0; k < rd_plan::kSide; ++k) {
        if (p->side[k]) cudaStreamDestroy(p->side[k]);
        if (p->join[k]) cudaEventDestroy(p->join[k]);
    }
    if (p->fork) cudaEventDestroy(p->fork);
    delete p;
}

extern "C" int rd_plan_create(const rd_fleet *f, int R, const int *robot, const int *kind,
                              int dtype, rd_plan **out)
{
    g_rd_error.clear();
    if (!out) return rd_fail(RD_ERR_ARG, "rd_plan_create: out is null");
    *out = nullptr;
    if (!f || !robot || !kind) return rd_fail(RD_ERR_ARG, "rd_plan_create: null argument");
    if (R < 1) return rd_fail(RD_ERR_RANGE, "rd_plan_create: R = %d", R);
    if (dtype != RD_F32 && dtype != RD_F64) return rd_fail(RD_ERR_DTYPE, "rd_plan_create: dtype %d", dtype);
    const size_t esz = dtype == RD_F32 ? 4 : 8;
    std::vector<long long> off(R);
    long long tot = 0;
    for (int r = 0; r < R; ++r) {
        if (robot[r] < 0 || robot[r] >= f->nrobots)
            return rd_fail(RD_ERR_ARG, "rd_plan_create: request %d names robot %d", r, robot[r]);
        if (kind[r] != RD_REQ_ID && kind[r] != RD_REQ_FD)
            return rd_fail(RD_ERR_ARG, "rd_plan_create: request %d has kind %d", r, kind[r]);
        off[r] = tot;
        tot += f->n[robot[r]];
    }
    // forward dynamics first (heavier), then longer chains first
    std::vector<int> order(R);
    std::iota(order.begin(), order.end(), 0);
    std::stable_sort(order.begin(), order.end(), [&](int a, int b) {
        if (kind[a] != kind[b]) return kind[a] > kind[b];
        return f->n[robot[a]] > f->n[robot[b]];
    });
    // forward-dynamics workspace per group of 32 sorted positions, laid out
    // [link][component][lane] so that a warp's accesses coalesce; sized by the
    // group's longest forward-dynamics chain. In FP32 plans a group whose
    // longest chain exceeds RD_ABA_EXTENDED_BIAS_LINKS runs its bias sweeps in
    // double-float (8 pairs per link instead of 10 scalars); being sorted
    // first, such groups form a prefix.
    const int groups32 = (R + 31) / 32;
    std::vector<long long> gws(groups32, 0), gwz(groups32, 0);
    std::vector<int> group_fd_n(groups32, 0);
    size_t ws = 0;
    int ext_groups = 0;
    for (int g = 0; g < groups32; ++g) {
        size_t nmax = 0;
        for (int k = 32 * g; k < R && k < 32 * g + 32; ++k)
            if (kind[order[k]] == RD_REQ_FD) nmax = std::max(nmax, (size_t)f->n[robot[order[k]]]);
        group_fd_n[g] = kind[order[32 * g]] == RD_REQ_FD ? (int)nmax : 0;
        if (!nmax) continue;
        const bool ext = dtype == RD_F32 && nmax > RD_ABA_EXTENDED_BIAS_LINKS;
        if (ext) ext_groups = g + 1;
        gws[g] = (long long)ws;
        ws += (nmax * (ext ? 16 : 10) * 32 * esz + 255) & ~(size_t)255;
        gwz[g] = (long long)ws;
        ws += (nmax * 8 * 32 * 8 + 255) & ~(size_t)255;
    }
    rd_plan *p = new (std::nothrow) rd_plan();
    if (!p) return rd_fail(RD_ERR_ALLOC, "rd_plan_create: host allocation failed");
    p->fleet = f;
    p->dtype = dtype;
    p->R = R;
    p->total_joints = tot;
    p->off = off;
    for (int k = 0; k < R;) {
        int j = k;
        const int r0 = order[k];
        while (j < R && kind[order[j]] == kind[r0] && f->n[robot[order[j]]] == f->n[robot[r0]]) ++j;
        p->groups.emplace_back(k, j);
        k = j;
    }
    cudaError_t e = cudaDeviceGetAttribute(&p->sms, cudaDevAttrMultiProcessorCount, f->device);
    if (e == cudaSuccess) e = upload(&p->order, order.data(), order.size());
    if (e == cudaSuccess) e = upload(&p->req_robot, robot, (size_t)R);
    if (e == cudaSuccess) e = upload(&p->req_kind, kind, (size_t)R);
    if (e == cudaSuccess) e = upload(&p->req_off, off.data(), off.size());
    if (e == cudaSuccess) e = upload(&p->group_ws, gws.data(), gws.size());
    if (e == cudaSuccess) e = upload(&p->group_wz, gwz.data(), gwz.size());
    if (e == cudaSuccess) e = cudaMalloc(&p->counter, 2 * sizeof(int));  // + the pair counter
    if (e == cudaSuccess) e = cudaMalloc(&p->ws, std::max<size_t>(ws, 16));
    p->ws_bytes = ws;
    p->ext_groups = ext_groups;
    p->group_fd_n = group_fd_n;
    if (e == cudaSuccess) e = cudaEventCreateWithFlags(&p->fork, cudaEventDisableTiming);
    for (int k = 0; k < rd_plan::kSide && e == cudaSuccess; ++k) {
        e = cudaStreamCreateWithFlags(&p->side[k], cudaStreamNonBlocking);
        if (e == cudaSuccess) e = cudaEventCreateWithFlags(&p->join[k], cudaEventDisableTiming);
    }
    if (e != cudaSuccess) {
        rd_plan_destroy(p);
        return rd_fail(RD_ERR_ALLOC, "rd_plan_create: %s", cudaGetErrorString(e));
    }
    *out = p;
    return RD_OK;
}

extern "C" long long rd_plan_total_joints(const rd_plan *p) { return p ? p->total_joints : -1; }

extern "C" int rd_plan_offsets(const rd_plan *p, long long *off)
{
    if (!p || !off) return rd_fail(RD_ERR_ARG, "rd_plan_offsets: null argument");
    std::copy(p->off.begin(), p->off.end(), off);
    return RD_OK;
}

extern "C" int rd_plan_groups(const rd_plan *p) { return p ? (int)p->groups.size() : -1; }

namespace {

// pair_n > 0: forward-dynamics groups whose first chain has at least pair_n
// links run two warps per 32 requests (fleet_pair_kernel), or three with
// three_warps (fleet_tri_kernel)
template <typename T, typename D>
int run_fleet(const rd_plan *p, const void *q, const void *qd, const void *in2, void *out,
              const double *b18, int *status, int schedule, int tune, int pair_n,
              bool three_warps, cudaStream_t s)
{
    const rd_fleet *f = p->fleet;
    rdyn::FleetArgs<T, D> a;
    if constexpr (sizeof(T) == 4) {
        a.consts = f->c32;
        a.robot_tn = f->tn32;
        a.robot_gb = f->gb32;
    } else {
        a.consts = f->c64;
        a.robot_tn = f->tn64;
        a.robot_gb = f->gb64;
    }
    if constexpr (std::is_same<D, double>::value) a.records = f->aba64;
    else a.records = f->abadf;
    a.records_df = f->abadf;
    a.ext_groups = p->ext_groups;
    a.pair_groups = 0;
    a.pair_counter = p->counter + 1;
    a.robot_n = f->robot_n;
    a.robot_link = f->robot_link;
    a.order = p->order;
    a.req_robot = p->req_robot;
    a.req_kind = p->req_kind;
    a.req_off = p->req_off;
    a.group_ws = p->group_ws;
    a.group_wz = p->group_wz;
    a.R = p->R;
    a.q = static_cast<const T *>(q);
    a.qd = static_cast<const T *>(qd);
    a.in2 = static_cast<const T *>(in2);
    a.out = static_cast<T *>(out);
    a.status = status;
    a.ws = p->ws;
    a.counter = p->counter;
    for (int k = 0; k < 6; ++k) {
        a.base.V0[k] = (T)b18[k];
        a.base.dV0[k] = (T)b18[6 + k];
        a.base.Fn[k] = (T)b18[12 + k];
    }
    cudaError_t e = cudaSuccess;
    if (schedule == RD_SCHED_PERSISTENT && pair_n > 0) {
        // two-warp forward dynamics for the leading groups whose first request
        // is a forward-dynamics chain of at least pair_n links
        int pg = 0;
        while (pg < (int)p->group_fd_n.size() && p->group_fd_n[pg] >= pair_n) ++pg;
        a.pair_groups = pg;
        int threads = (tune >> 8) & 0xff ? 1 << ((tune >> 8) & 0xff) : 128;
        int per_sm = tune & 0xff ? tune & 0xff : 4;
        if (three_warps) {
            // 2^t threads name 2^t / 64 groups per block, as for pairs: 1 or 2
            if (threads != 64 && threads != 128)
                return rd_fail(RD_ERR_ARG, "fleet_batch: the three-warp schedule takes one or two "
                                           "triples per block (tune threads 64 or 128, got %d)",
                               threads);
            threads = 96 * (threads / 64);
        } else if (threads < 64 || threads > 448 || threads % 64) {
            return rd_fail(RD_ERR_ARG, "fleet_batch: the two-warp schedule takes 64..448 threads "
                                       "per block in multiples of 64 (%d)", threads);
        }
        e = cudaMemsetAsync(p->counter, 0, 2 * sizeof(int), s);
        if (e != cudaSuccess) return rd_cuda_fail(e, "fleet_batch: counter reset");
        if (three_warps)
            rdyn::fleet_tri_kernel<T, D><<<p->sms * per_sm, threads, 0, s>>>(a);
        else
            rdyn::fleet_pair_kernel<T, D><<<p->sms * per_sm, threads, 0, s>>>(a);
    } else if (schedule == RD_SCHED_PERSISTENT) {
        int threads = (tune >> 8) & 0xff ? 1 << ((tune >> 8) & 0xff) : 128;
        int per_sm = tune & 0xff ? tune & 0xff : 4;
        if (threads < 32 || threads > 1024)
            return rd_fail(RD_ERR_ARG, "fleet_batch: %d threads per block", threads);
        e = cudaMemsetAsync(p->counter, 0, sizeof(int), s);
        if (e != cudaSuccess) return rd_cuda_fail(e, "fleet_batch: counter reset");
        rdyn::fleet_persistent_kernel<T, D><<<p->sms * per_sm, threads, 0, s>>>(a);
    } else if (schedule == RD_SCHED_PER_GROUP) {
        // one launch per group, spread over side streams that fork from and
        // join back into the caller's stream (so groups can run concurrently)
        e = cudaEventRecord(p->fork, s);
        for (int k = 0; k < rd_plan::kSide && e == cudaSuccess; ++k)
            e = cudaStreamWaitEvent(p->side[k], p->fork, 0);
        if (e != cudaSuccess) return rd_cuda_fail(e, "fleet_batch: fork");
        int k = 0;
        for (const auto &g : p->groups) {
            const int len = g.second - g.first;
            rdyn::fleet_range_kernel<T, D><<<(len + 127) / 128, 128, 0, p->side[k]>>>(a, g.first, g.second);
            k = (k + 1) % rd_plan::kSide;
        }
        for (int j = 0; j < rd_plan::kSide && e == cudaSuccess; ++j) {
            e = cudaEventRecord(p->join[j], p->side[j]);
            if (e == cudaSuccess) e = cudaStreamWaitEvent(s, p->join[j], 0);
        }
        if (e != cudaSuccess) return rd_cuda_fail(e, "fleet_batch: join");
    } else {
        return rd_fail(RD_ERR_ARG, "fleet_batch: unknown schedule %d", schedule);
    }
    e = cudaGetLastError();
    if (e != cudaSuccess) return rd_cuda_fail(e, "fleet_batch launch");
    return RD_OK;
}

}  // namespace

extern "C" int fleet_batch(const rd_plan *p, const void *q, const void *qd, const void *in2,
                           void *out, const double *base, int *status, int schedule, int tune,
                           void *stream)
{
    g_rd_error.clear();
    if (!p) return rd_fail(RD_ERR_ARG, "fleet_batch: null plan");
    if (!q || !qd || !in2 || !out) return rd_fail(RD_ERR_ARG, "fleet_batch: null data pointer");
    if (out == q || out == qd || out == in2)
        return rd_fail(RD_ERR_ARG, "fleet_batch: out aliases an input");
    static const double dflt[18] = {0, 0, 0, 0, 0, 0, 0, 0, 9.81, 0, 0, 0, 0, 0, 0, 0, 0, 0};
    const double *b18 = base ? base : dflt;
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    const bool fp64_update = (schedule & RD_FLEET_FP64_UPDATE) != 0;
    schedule &= ~RD_FLEET_FP64_UPDATE;
    const int pair_n = (tune >> 16) & 0xff;
    const bool three = ((tune >> 24) & 1) != 0;
    if ((pair_n || three) && schedule != RD_SCHED_PERSISTENT)
        return rd_fail(RD_ERR_ARG, "fleet_batch: two- or three-warp forward dynamics needs the "
                                   "persistent schedule");
    if (three && !pair_n)
        return rd_fail(RD_ERR_ARG, "fleet_batch: RD_FLEET_THREE_WARPS needs a chain length");
    if (p->dtype == RD_F32) {
        if (fp64_update)
            return run_fleet<float, double>(p, q, qd, in2, out, b18, status, schedule, tune, pair_n,
                                            three, s);
        return run_fleet<float, rdyn::DF>(p, q, qd, in2, out, b18, status, schedule, tune, pair_n,
                                          three, s);
    }
    return run_fleet<double, double>(p, q, qd, in2, out, b18, status, schedule, tune, pair_n,
                                     three, s);
}
