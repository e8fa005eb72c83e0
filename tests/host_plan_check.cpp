// Invariants of the host tier's step plan (paper_2509_15645_b300/csrc/host_plan.hpp),
// checked over random sequences of chunk-touch maps: prints "ok" and exits 0, or
// names the first violated invariant and exits 1.
#include <cstdio>
#include <cstdlib>
#include <random>
#include <set>
#include <vector>

#include "host_plan.hpp"

using namespace gs;

static int fails = 0;
#define CHECK(cond, ...)                                                   \
    do {                                                                   \
        if (!(cond)) {                                                     \
            if (fails++ < 10) {                                            \
                std::printf("FAIL %s:%d ", __FILE__, __LINE__);            \
                std::printf(__VA_ARGS__);                                  \
                std::printf("\n");                                         \
            }                                                              \
        }                                                                  \
    } while (0)

// Chunks covered by runs [lo, hi), each exactly once, with consecutive slots.
static std::vector<int> covered(const HostPlan &P, size_t lo, size_t hi, int64_t nch)
{
    std::vector<int> seen(nch, 0);
    for (size_t k = lo; k < hi; k++) {
        const HostRun &r = P.runs[k];
        CHECK(r.nchunks >= 1, "empty run");
        for (int64_t j = 0; j < r.nchunks; j++) {
            const int64_t ch = r.chunk0 + j;
            CHECK(ch >= 0 && ch < nch, "run chunk out of range");
            if (ch < 0 || ch >= nch) continue;
            CHECK(P.slot[ch] == r.slot0 + j, "run slot mismatch at chunk %lld", (long long)ch);
            seen[ch]++;
        }
    }
    return seen;
}

int main()
{
    std::mt19937_64 rng(12345);
    int steps_half = 0, steps_full = 0, steps_reuse = 0, druns_seen = 0, late_rounds = 0, multi_rounds = 0;
    for (int scenario = 0; scenario < 400; scenario++) {
        const int64_t nch = 1 + rng() % 200;
        const int64_t stage = 1 + rng() % 160;
        HostHistory h;
        h.reset(nch);
        // a "view" is a window of chunks; consecutive steps overlap partly
        int64_t centre = rng() % nch;
        for (int step = 0; step < 12; step++) {
            std::vector<uint8_t> touch(nch, 0);
            const int64_t width = 1 + rng() % std::max<int64_t>(1, nch / 3);
            centre = (centre + (int64_t)(rng() % (2 * width + 1)) - width + nch) % nch;
            for (int64_t j = 0; j < width; j++) touch[(centre + j) % nch] = 2;
            const int pu = (int)(rng() % 100);
            for (int64_t ch = 0; ch < nch; ch++)
                if (!touch[ch] && (int)(rng() % 100) < pu / 3) touch[ch] = 1;
            const HostPlan P = plan_host_step(touch.data(), nch, stage, h);
            int64_t nv = 0, nu = 0;
            for (auto t : touch) nv += t == 2, nu += t == 1;
            CHECK(P.nv == nv && P.nu == nu, "counts");
            const int64_t H = stage / 2;
            const bool fits_half = H >= 1 && nv <= H && (nu == 0 || H - nv >= 1);
            CHECK(P.half == fits_half, "half-mode choice");
            const bool fits = nv <= stage && (nu == 0 || stage - nv >= 1);
            if (!P.ok) {
                CHECK(!fits, "refused a step that fits the ring");
                h.reset(nch);
                continue;
            }
            CHECK(fits, "accepted a step that does not fit the ring");
            CHECK(P.reuse == (P.half && !h.prev_full), "reuse only in half mode after a half-mode step");
            steps_half += P.half, steps_full += !P.half, steps_reuse += P.reuse;
            const int64_t base = P.half ? P.p * H : 0, ring = P.half ? H : stage;
            if (P.half) CHECK(P.p == h.parity, "half follows the parity");
            // slots: untouched -1; visible chunks first, in order; all inside the ring (half)
            int64_t q = 0;
            for (int64_t ch = 0; ch < nch; ch++) {
                if (touch[ch] == 0) CHECK(P.slot[ch] == -1, "untouched chunk has a slot");
                if (touch[ch] == 2) {
                    CHECK(P.slot[ch] == base + q, "visible slot order");
                    q++;
                }
                if (touch[ch] == 1)
                    CHECK(P.slot[ch] >= base + nv && P.slot[ch] < base + ring, "round slot outside its area");
                if (touch[ch]) CHECK(P.slot[ch] >= 0 && P.slot[ch] < stage, "slot outside the ring");
            }
            // rounds: contiguous chunk ranges covering [0, nch); distinct slots within a round;
            // rounds k and k+1 use disjoint slots when there are two sub-halves
            CHECK(!P.rounds.empty() && P.rounds.front().ch_lo == 0 && P.rounds.back().ch_hi == nch, "round span");
            std::vector<std::set<int32_t>> rslots(P.rounds.size());
            for (size_t k = 0; k < P.rounds.size(); k++) {
                const HostRound &r = P.rounds[k];
                if (k) CHECK(r.ch_lo == P.rounds[k - 1].ch_hi, "rounds not contiguous");
                int64_t in_round = 0;
                bool late = false;
                for (int64_t ch = r.ch_lo; ch < r.ch_hi; ch++) {
                    if (touch[ch] != 1) continue;
                    in_round++;
                    late |= h.pstaged[ch] != 0;
                    CHECK(rslots[k].insert(P.slot[ch]).second, "two chunks of a round share a slot");
                }
                CHECK(in_round <= P.rcap, "round larger than rcap");
                CHECK(r.late == late, "late flag of a round");
                late_rounds += r.late;
                // its runs cover exactly its visible chunks and its optimizer-only chunks
                auto sv = covered(P, r.vis_lo, r.vis_hi, nch);
                auto su = covered(P, r.upd_lo, r.upd_hi, nch);
                for (int64_t ch = 0; ch < nch; ch++) {
                    const bool inr = ch >= r.ch_lo && ch < r.ch_hi;
                    CHECK(sv[ch] == (inr && touch[ch] == 2 ? 1 : 0), "round write-back runs");
                    CHECK(su[ch] == (inr && touch[ch] == 1 ? 1 : 0), "round optimizer runs");
                }
            }
            multi_rounds += P.rounds.size() > 1;
            if (P.nbuf == 2)
                for (size_t k = 0; k + 1 < P.rounds.size(); k++)
                    for (int32_t sl : rslots[k]) CHECK(!rslots[k + 1].count(sl), "consecutive rounds share a slot");
            for (int32_t sl : (P.rounds.empty() ? std::set<int32_t>() : rslots[0]))
                CHECK(sl >= base + nv, "round slot over a visible slot");
            // visible chunks: each from exactly one source (device copy, host now, host late)
            auto now = covered(P, P.now_lo, P.late_lo, nch);
            auto late = covered(P, P.late_lo, P.late_hi, nch);
            std::vector<int> dev(nch, 0);
            for (const auto &d : P.druns) {
                druns_seen++;
                CHECK(P.reuse, "device copies without reuse");
                for (int64_t j = 0; j < d[2]; j++) {
                    const int64_t dst = d[1] + j;
                    int64_t ch = -1;
                    for (int64_t c2 = 0; c2 < nch; c2++)
                        if (touch[c2] == 2 && P.slot[c2] == dst) ch = c2;
                    CHECK(ch >= 0, "device copy to a slot no visible chunk holds");
                    if (ch < 0) continue;
                    CHECK(h.pvslot[ch] == d[0] + j, "device copy from a slot the chunk did not hold");
                    // the source lies in the other half: this step's H2D and copies never write it
                    CHECK(d[0] + j < (1 - P.p) * H + H && d[0] + j >= (1 - P.p) * H, "device copy source in this half");
                    dev[ch]++;
                }
            }
            for (int64_t ch = 0; ch < nch; ch++) {
                if (touch[ch] != 2) {
                    CHECK(now[ch] + late[ch] + dev[ch] == 0, "non-visible chunk in the visible H2D");
                    continue;
                }
                CHECK(now[ch] + late[ch] + dev[ch] == 1, "visible chunk %lld sourced %d times", (long long)ch,
                      now[ch] + late[ch] + dev[ch]);
                if (dev[ch]) CHECK(h.pvslot[ch] >= 0, "copied chunk was not visible before");
                if (now[ch]) CHECK(!h.pstaged[ch], "chunk staged by the previous step read from the host at once");
                if (late[ch]) CHECK(h.pstaged[ch], "late chunk was not staged before");
            }
            advance_host_history(h, touch.data(), nch, P);
            for (int64_t ch = 0; ch < nch; ch++) {
                CHECK(h.pvslot[ch] == (touch[ch] == 2 ? P.slot[ch] : -1), "history slots");
                CHECK(h.pstaged[ch] == (touch[ch] != 0), "history staged");
            }
            CHECK(h.prev_full == !P.half, "history mode");
        }
    }
    std::printf("half %d full %d reuse %d device-copy runs %d late rounds %d multi-round %d\n", steps_half,
                steps_full, steps_reuse, druns_seen, late_rounds, multi_rounds);
    if (!steps_half || !steps_full || !steps_reuse || !druns_seen || !late_rounds || !multi_rounds) {
        std::printf("FAIL coverage\n");
        return 1;
    }
    if (fails) return 1;
    std::printf("ok\n");
    return 0;
}
