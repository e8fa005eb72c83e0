// host_plan.hpp -- the host tier's per-step plan (§4.2 selective offloading):
// which staging-ring slot each touched chunk of SH rows takes, where its rows
// come from, the rounds in which the optimizer-only chunks pass through the
// ring, and the copy runs.  Plain C++ (no CUDA): gs_runtime.cu enqueues the
// copies and kernels the plan describes, and a CPU test checks its invariants.
#pragma once

#include <array>
#include <cstdint>
#include <vector>

namespace gs {

// Chunks [chunk0, chunk0 + nchunks) in slots [slot0, slot0 + nchunks).
struct HostRun {
    int64_t chunk0, slot0, nchunks;
};

// Optimizer round: the update-set members with ids in chunks [ch_lo, ch_hi);
// runs [vis_lo, vis_hi) write back the visible chunks of that range after the
// round's apply, runs [upd_lo, upd_hi) bring in and write back its
// optimizer-only chunks; `late`: one of those was staged by the previous step,
// so their H2D waits for its write-backs.
struct HostRound {
    int64_t ch_lo, ch_hi;
    size_t vis_lo, vis_hi, upd_lo, upd_hi;
    bool late;
};

// What a step leaves for the next: each chunk's slot if it was visible (its
// slot holds its final rows until the step after next), whether it was staged
// at all, the ring half the next step takes, whether this step used the whole
// ring (or there was no step).
struct HostHistory {
    std::vector<int32_t> pvslot;
    std::vector<uint8_t> pstaged;
    int parity = 0;
    bool prev_full = true;
    void reset(int64_t nch)
    {
        pvslot.assign(nch, -1);
        pstaged.assign(nch, 0);
        parity = 0;
        prev_full = true;
    }
};

struct HostPlan {
    bool ok = false;               // false: the visible chunks (plus one round slot) exceed the ring
    int64_t nv = 0, nu = 0;        // visible chunks, optimizer-only chunks
    bool half = false;             // the step uses half `p` of the ring
    int p = 0;
    bool reuse = false;            // visible chunks of the previous step are copied on the device
    int64_t nbuf = 1, rcap = 1;    // optimizer rounds: ring sub-halves, chunks per round
    std::vector<int32_t> slot;     // chunk -> slot, -1 if not staged
    std::vector<HostRun> runs;     // [now_lo, late_lo) H2D at once, [late_lo, late_hi) H2D after the
    size_t now_lo = 0, late_lo = 0, late_hi = 0;   // previous write-backs; then the rounds' runs
    std::vector<HostRound> rounds;
    std::vector<std::array<int64_t, 3>> druns;     // device copies {source slot, destination slot, chunks}
};

// touch[ch]: 2 = a visible Gaussian in chunk ch, 1 = only optimizer members, 0 = untouched.
// A step whose chunks fit in half of the ring (the visible ones plus at least
// one round slot) takes the half the previous step did not: its H2D then need
// not wait for the previous step's write-backs, the chunks the previous step
// had visible are copied from their slots on the device, and those it staged
// only for the optimizer come from the host after its write-backs.  Otherwise
// the whole ring, after every write-back.  Visible chunks take the first
// slots of the ring (or half) in chunk order; optimizer-only chunks go through
// the rest in rounds of at most `rcap` chunks cut at chunk-id boundaries,
// alternating between two sub-halves.
inline HostPlan plan_host_step(const uint8_t *touch, int64_t nch, int64_t stage_chunks, const HostHistory &h)
{
    HostPlan P;
    for (int64_t ch = 0; ch < nch; ch++) {
        if (touch[ch] == 2) P.nv++;
        else if (touch[ch] == 1) P.nu++;
    }
    const int64_t H = stage_chunks / 2;
    P.half = H >= 1 && P.nv <= H && (P.nu == 0 || H - P.nv >= 1);
    P.p = P.half ? h.parity : 0;
    const int64_t base = P.half ? P.p * H : 0, ring_chunks = P.half ? H : stage_chunks;
    P.reuse = P.half && !h.prev_full;
    const int64_t cap = ring_chunks - P.nv;
    if (P.nv > stage_chunks || (P.nu > 0 && cap < 1)) return P;
    P.ok = true;
    P.slot.assign(nch, -1);
    {
        int64_t q = 0;
        for (int64_t ch = 0; ch < nch; ch++)
            if (touch[ch] == 2) P.slot[ch] = (int32_t)(base + q++);
    }
    P.nbuf = cap >= 2 ? 2 : 1;
    P.rcap = P.nu > 0 ? cap / P.nbuf : 1;
    {
        HostRound r{0, nch, 0, 0, 0, 0, false};
        int64_t in_round = 0;
        for (int64_t ch = 0; ch < nch; ch++) {
            if (touch[ch] != 1) continue;
            if (in_round == P.rcap) {          // close the round before this chunk
                r.ch_hi = ch;
                P.rounds.push_back(r);
                r = HostRound{ch, nch, 0, 0, 0, 0, false};
                in_round = 0;
            }
            P.slot[ch] = (int32_t)(base + P.nv + ((int64_t)P.rounds.size() % P.nbuf) * P.rcap + in_round);
            r.late |= h.pstaged[ch] != 0;
            in_round++;
        }
        P.rounds.push_back(r);
    }
    auto add_run = [&](int64_t ch, size_t first) {
        const int64_t s = P.slot[ch];
        if (P.runs.size() > first && P.runs.back().chunk0 + P.runs.back().nchunks == ch &&
            P.runs.back().slot0 + P.runs.back().nchunks == s)
            P.runs.back().nchunks++;
        else
            P.runs.push_back(HostRun{ch, s, 1});
    };
    // visible chunks by source: 0 device copy, 1 host rows now, 2 host rows
    // after the previous write-backs
    auto src_class = [&](int64_t ch) {
        if (P.reuse && h.pvslot[ch] >= 0) return 0;
        return h.pstaged[ch] ? 2 : 1;
    };
    for (int64_t ch = 0; ch < nch; ch++) {
        if (touch[ch] != 2 || src_class(ch) != 0) continue;
        const int64_t src = h.pvslot[ch], dst = P.slot[ch];
        if (!P.druns.empty() && P.druns.back()[0] + P.druns.back()[2] == src &&
            P.druns.back()[1] + P.druns.back()[2] == dst)
            P.druns.back()[2]++;
        else
            P.druns.push_back({src, dst, 1});
    }
    P.now_lo = P.runs.size();
    for (int64_t ch = 0; ch < nch; ch++)
        if (touch[ch] == 2 && src_class(ch) == 1) add_run(ch, P.now_lo);
    P.late_lo = P.runs.size();
    for (int64_t ch = 0; ch < nch; ch++)
        if (touch[ch] == 2 && src_class(ch) == 2) add_run(ch, P.late_lo);
    P.late_hi = P.runs.size();
    for (HostRound &r : P.rounds) {           // visible chunks again, for the write-backs
        r.vis_lo = P.runs.size();
        for (int64_t ch = r.ch_lo; ch < r.ch_hi; ch++)
            if (touch[ch] == 2) add_run(ch, r.vis_lo);
        r.vis_hi = P.runs.size();
    }
    for (HostRound &r : P.rounds) {           // optimizer-only chunks
        r.upd_lo = P.runs.size();
        for (int64_t ch = r.ch_lo; ch < r.ch_hi; ch++)
            if (touch[ch] == 1) add_run(ch, r.upd_lo);
        r.upd_hi = P.runs.size();
    }
    return P;
}

// The history the next step plans with.
inline void advance_host_history(HostHistory &h, const uint8_t *touch, int64_t nch, const HostPlan &P)
{
    for (int64_t ch = 0; ch < nch; ch++) {
        h.pvslot[ch] = touch[ch] == 2 ? P.slot[ch] : -1;
        h.pstaged[ch] = touch[ch] != 0;
    }
    h.prev_full = !P.half;
    if (P.half) h.parity ^= 1;
}

}  // namespace gs
