// kerr_trace_x2.cuh -- the FP32 stepping phase with two geodesics per thread.
//
// Each thread holds two geodesics ("slots") and advances both with one
// instruction stream: the right-hand sides and RK4 stages of an attempt run
// on packed f32x2 instructions (kerr_f2.cuh), so a warp issues about half the
// FP32 arithmetic instructions per geodesic of the one-per-thread kernel.
// Everything that branches per geodesic -- the error measure, step control,
// compensated update, termination events, crossings, renormalisation -- runs
// per slot in scalar FP32 (or FP64) code,
// the same functions the one-per-thread kernel calls, so a geodesic's
// arithmetic is that of the one-per-thread kernel with out-of-line
// right-hand sides.  Work distribution as in trace_f32_kernel (phase 0): idle
// slots refill from the atomic queue (one warp-aggregated claim per slot and
// warp), geodesics entering the FP64 zone are deferred to the zone phase.
#pragma once

#include "kerr_f2.cuh"
#include "kerr_trace.cuh"

namespace kerr {

__device__ __forceinline__ float slot_get(const f2 &v, int s) { return s == 0 ? v.v.x : v.v.y; }
__device__ __forceinline__ void slot_put(f2 &v, int s, float x)
{
    if (s == 0)
        v.v.x = x;
    else
        v.v.y = x;
}

// The FP32 constants of a slot (the FP64 ones are loaded when needed).
struct SlotConst {
    float af, rcapf, rescf, zonef, tendf, tendlo;
    int flags;
};

__device__ __forceinline__ void load_slot_const(const TraceParams &P, int64_t id, SlotConst &k)
{
    const int64_t n = P.n;
    k.af = P.s_const[KC_A * n + id];
    k.rcapf = P.s_const[KC_RCAP * n + id];
    k.rescf = P.s_const[KC_RESC * n + id];
    k.zonef = P.s_const[KC_ZONE * n + id];
    k.tendf = P.s_const[KC_TEND * n + id];
    k.tendlo = P.s_const[KC_TENDLO * n + id];
    k.flags = __float_as_int(P.s_const[KC_FLAGS * n + id]);
}

__device__ __forceinline__ RayConst slot_rc(const SlotConst &k)
{
    RayConst rc;
    rc.af = k.af;
    rc.rcapf = k.rcapf;
    rc.rescf = k.rescf;
    rc.zonef = k.zonef;
    rc.tendf = k.tendf;
    rc.tendlo = k.tendlo;
    rc.use_t = k.flags & 1;
    rc.tpos = (k.flags >> 1) & 1;
    return rc;
}

template <int BLOCK, int MINB>
__global__ void __launch_bounds__(BLOCK, MINB) trace_f32x2_kernel(const TraceParams P)
{
    constexpr int RM = RHS_CALL;
    const unsigned FULL = 0xffffffffu;
    const int lane = threadIdx.x & 31;
    const unsigned lt_mask = (1u << lane) - 1u;
    const int64_t n = P.n;
    unsigned long long n_items = (unsigned long long)n;
    if (P.n_dev && *P.n_dev < n_items)
        n_items = *P.n_dev;
    const unsigned long long zcap = (unsigned long long)P.zcap;
    const bool can_defer = P.zbuf != nullptr && P.fp64_zone > 0.0;
    const float tol = (float)P.tol;
    const float h0 = (float)P.h0;

    bool has[2] = {false, false};
    bool drained = false, timed_out = false;
    int64_t id[2] = {0, 0};
    SlotConst rc[2];
    f2 y[8], c[8];
#pragma unroll
    for (int i = 0; i < 8; ++i) {
        y[i] = f2(0.f, 0.f);
        c[i] = f2(0.f, 0.f);
    }
    rc[0].af = rc[1].af = 0.f;
    float h[2] = {0.f, 0.f}, rnow[2] = {0.f, 0.f};
    uint32_t nsteps[2] = {0, 0};
    int since_renorm[2] = {0, 0};
    Counters C;
    const unsigned long long t_start = global_ns();
    uint32_t iter = 0;

    for (;;) {
        // ---- refill idle slots from the queue (one atomic per slot and warp)
#pragma unroll
        for (int s = 0; s < 2; ++s) {
            const unsigned need = __ballot_sync(FULL, !has[s]);
            if (need && !drained) {
                const unsigned long long base = warp_claim(P.head, need);
                if (base + __popc(need) >= n_items)
                    drained = true;
                const unsigned long long my = base + __popc(need & lt_mask);
                if (!has[s] && my < n_items) {
                    const int64_t g = (int64_t)my;
                    if (P.status[g] == ST_NONE) {     // set-up may have ended it
                        id[s] = g;
#pragma unroll
                        for (int i = 0; i < 8; ++i) {
                            slot_put(y[i], s, P.s_state[i * n + g]);
                            slot_put(c[i], s, P.s_state[(8 + i) * n + g]);
                        }
                        load_slot_const(P, g, rc[s]);
                        h[s] = h0;
                        nsteps[s] = 0;
                        since_renorm[s] = 0;
                        rnow[s] = ks_r(rc[s].af * rc[s].af, slot_get(y[1], s), slot_get(y[2], s),
                                       slot_get(y[3], s));
                        if (timed_out) {
                            P.status[g] = ST_TIMEOUT;
                            P.steps[g] = 0;
                            C.status(ST_TIMEOUT);
                        } else {
                            has[s] = true;
                        }
                    }
                }
            }
        }
        if (!__any_sync(FULL, has[0] || has[1])) {
            if (drained)
                break;
            continue;
        }
        // ---- zone entries: defer them to the zone phase
        bool in_zone[2];
#pragma unroll
        for (int s = 0; s < 2; ++s) {
            in_zone[s] = has[s] && rnow[s] < rc[s].zonef;
            if (can_defer) {
                const bool want = in_zone[s] && !timed_out;
                const unsigned dm = __ballot_sync(FULL, want);
                if (dm) {
                    const unsigned long long zb = warp_claim(P.zcount, dm);
                    if (want) {
                        const unsigned long long slot = zb + __popc(dm & lt_mask);
                        if (slot < zcap) {
                            ZoneEntry &e = P.zbuf[slot];
#pragma unroll
                            for (int i = 0; i < 8; ++i) {
                                e.y[i] = slot_get(y[i], s);
                                e.c[i] = slot_get(c[i], s);
                            }
                            e.id = id[s];
                            e.h = h[s];
                            e.rnow = rnow[s];
                            e.nsteps = nsteps[s];
                            e.since_renorm = since_renorm[s];
                            e.fmt = ZE_PAIR;
                            e.seq = (uint32_t)(slot + 1ull);   // visible to the next launch
                            ++C.def;
                            has[s] = false;
                            in_zone[s] = false;
                        }
                    }
                }
            }
        }
        // ---- per-slot checks
        int st[2] = {ST_NONE, ST_NONE};
        bool fp32_step[2] = {false, false};
        ClipRec cr[2];
#pragma unroll
        for (int s = 0; s < 2; ++s) {
            if (!has[s])
                continue;
            if (timed_out) {
                st[s] = ST_TIMEOUT;
            } else if ((int64_t)nsteps[s] >= P.max_steps) {
                st[s] = ST_MAXSTEPS;
            } else {
                ++nsteps[s];
                ++C.att;
                // a geodesic inside the zone is always deferred (the zone
                // buffer holds one entry per geodesic); one that could not be
                // would be counted and step in FP32
                if (in_zone[s])
                    C.status(ST_NONE);
                fp32_step[s] = true;
            }
        }
        // ---- one packed attempt for the slots stepping in FP32 (an idle
        // slot's half computes on stale registers and is discarded)
        if (fp32_step[0] || fp32_step[1]) {
            const f2 av(rc[0].af, rc[1].af);
            const f2 a2 = av * av;
            const f2 hv(h[0], h[1]);
            f2 A0[4], d[8], df[8];
            rhs<RM>(av, a2, y[1], y[2], y[3], y[4], y[5], y[6], y[7], A0);
            rk4_incr<RM>(av, a2, y, A0, hv, df);
            two_halves<RM>(av, a2, y, A0, hv, d);
#pragma unroll
            for (int s = 0; s < 2; ++s) {
                if (!fp32_step[s])
                    continue;
                float ys[8], cs[8], ds[8], dfs[8], A0s[4];
#pragma unroll
                for (int i = 0; i < 8; ++i) {
                    ys[i] = slot_get(y[i], s);
                    cs[i] = slot_get(c[i], s);
                    ds[i] = slot_get(d[i], s);
                    dfs[i] = slot_get(df[i], s);
                }
#pragma unroll
                for (int j = 0; j < 4; ++j)
                    A0s[j] = slot_get(A0[j], s);
                const float err = err_norm_f(ys, ds, dfs, tol);
                uint32_t r = 11;
                st[s] = step_post<true, float, false, RM, true>(slot_rc(rc[s]), P, id[s], rc[s].af,
                                                                slot_get(a2, s), A0s, ds, err, ys,
                                                                cs, h[s], rnow[s], r, C.acc,
                                                                since_renorm[s], nullptr,
                                                                P.clipq ? &cr[s] : nullptr);
                C.rhs32 += r;
#pragma unroll
                for (int i = 0; i < 8; ++i) {
                    slot_put(y[i], s, ys[i]);
                    slot_put(c[i], s, cs[i]);
                }
            }
        }
        // ---- geodesics that ended (a deferred clip keeps the state before
        // the step and goes to the clip queue)
        bool p32[2] = {false, false};
#pragma unroll
        for (int s = 0; s < 2; ++s) {
            if (st[s] == ST_NONE)
                continue;
            const int64_t g = id[s];
#pragma unroll
            for (int i = 0; i < 8; ++i) {
                P.s_state[i * n + g] = slot_get(y[i], s);
                P.s_state[(8 + i) * n + g] = slot_get(c[i], s);
            }
            P.status[g] = st[s];
            P.steps[g] = (int32_t)nsteps[s];
            if (cr[s].pending) {
                P.clip_h[g] = h[s];
                P.clip_shi[g] = cr[s].s_hi;
                p32[s] = true;      // all steps of this kernel are FP32 steps
            }
            C.status(st[s]);
            has[s] = false;
        }
        if (P.clipq) {
#pragma unroll
            for (int s = 0; s < 2; ++s)
                enqueue_clips(P, p32[s], false, id[s]);
        }
        // ---- wall-time budget (warp-uniform decision)
        if ((P.budget_ns || P.abort) && ((++iter & 31u) == 0) && !timed_out) {
            bool over = false;
            if (lane == 0)
                over = stop_requested(P, t_start);
            timed_out = __shfl_sync(FULL, over, 0);
        }
    }
    C.flush(P.stats);
}

} // namespace kerr
