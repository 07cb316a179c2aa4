// Checks of the request server's admission policy (paper_2211_15383_gb300/csrc/admission.h),
// compiled and run by tests/test_serving_host.py.  Exit status 0 when every check holds;
// otherwise the failed check is printed.
#include <cstdio>
#include <cstdlib>
#include <map>
#include <random>
#include <vector>

#include "admission.h"

using mg::Admission;

static int failures = 0;
#define CHECK(cond)                                                   \
    do {                                                              \
        if (!(cond)) {                                                \
            std::printf("FAILED line %d: %s\n", __LINE__, #cond);    \
            ++failures;                                               \
        }                                                             \
    } while (0)

static std::vector<uint64_t> ids(const std::vector<Admission::Item>& v) {
    std::vector<uint64_t> out;
    for (auto& it : v) out.push_back(it.id);
    return out;
}

int main() {
    {   // first fit in arrival order, slots and budget respected
        Admission a(100, 2, 2);
        a.push(1, 60);
        a.push(2, 60);
        a.push(3, 30);
        a.push(4, 30);
        CHECK((ids(a.admit()) == std::vector<uint64_t>{1, 3}));   // 2 does not fit beside 1; 3 does
        CHECK(a.reserved() == 90 && a.active() == 2);
        CHECK(a.queue().front().id == 2 && a.queue().front().bypassed == 1);
        a.finish(60);                                              // 1 done
        CHECK((ids(a.admit()) == std::vector<uint64_t>{2}));       // 2 fits now; 4 waits for a slot
        a.finish(30);                                              // 3 done
        CHECK((ids(a.admit()) == std::vector<uint64_t>{4}));
        CHECK(a.max_reserved() <= 100 && a.max_active_seen() == 2);
    }
    {   // a large request is overtaken at most max_bypass times
        Admission a(100, 8, 2);
        a.push(1, 20);
        CHECK((ids(a.admit()) == std::vector<uint64_t>{1}));
        a.push(2, 90);                                             // does not fit beside 1
        CHECK(a.admit().empty());
        a.push(3, 20);
        CHECK((ids(a.admit()) == std::vector<uint64_t>{3}));       // overtakes 2 (1st time)
        a.push(4, 20);
        CHECK((ids(a.admit()) == std::vector<uint64_t>{4}));       // overtakes 2 (2nd time)
        a.push(5, 20);
        CHECK(a.admit().empty());                                  // 2 waits for no one else
        a.finish(20);
        a.finish(20);
        CHECK(a.admit().empty());                                  // 20 reserved: 2 still does not fit
        a.finish(20);
        CHECK((ids(a.admit()) == std::vector<uint64_t>{2}));       // 5 does not fit beside 2
        CHECK(a.queued() == 1 && a.queue().front().id == 5);
    }
    {   // equal sizes: strictly first in, first admitted
        Admission a(1000, 3, 4);
        std::vector<uint64_t> order;
        for (uint64_t i = 1; i <= 10; ++i) a.push(i, 100);
        while (a.queued() > 0 || a.active() > 0) {
            for (auto& it : a.admit()) order.push_back(it.id);
            if (a.active() > 0) a.finish(100);
        }
        for (size_t i = 0; i < order.size(); ++i) CHECK(order[i] == i + 1);
        CHECK(order.size() == 10);
    }
    {   // removal of a queued request; a request put back at the head blocks the others
        Admission a(100, 4, 4);
        a.push(1, 80);
        a.admit();
        a.push(2, 50);
        a.push(3, 10);
        CHECK(a.remove(2) && !a.remove(2));
        CHECK((ids(a.admit()) == std::vector<uint64_t>{3}));
        a.finish(80);
        a.push_front(7, 95);                                       // needs 95, 10 reserved
        a.push(8, 5);
        CHECK(a.admit().empty());                                  // 8 would fit, but 7 is not overtaken
        a.finish(10);
        CHECK((ids(a.admit()) == std::vector<uint64_t>{7, 8}));
        CHECK(a.too_large(101) && !a.too_large(100));
    }
    {   // random arrivals and completions: invariants, and every request admitted once
        std::mt19937_64 rng(12345);
        const size_t budget = 1000;
        const int max_active = 4, max_bypass = 3;
        Admission a(budget, max_active, max_bypass);
        std::map<uint64_t, size_t> running;
        std::map<uint64_t, int> admitted;
        uint64_t next = 1;
        for (int step = 0; step < 20000; ++step) {
            const int what = (int)(rng() % 3);
            if (what == 0 && next <= 3000) {
                a.push(next++, 1 + rng() % budget);
            } else if (what == 1 && !running.empty()) {
                auto it = running.begin();
                std::advance(it, (long)(rng() % running.size()));
                a.finish(it->second);
                running.erase(it);
            }
            for (auto& it : a.admit()) {
                running[it.id] = it.bytes;
                ++admitted[it.id];
            }
            size_t sum = 0;
            for (auto& kv : running) sum += kv.second;
            CHECK(sum == a.reserved() && a.reserved() <= budget);
            CHECK((int)running.size() == a.active() && a.active() <= max_active);
            for (auto& q : a.queue()) CHECK(q.bypassed <= max_bypass);
            if (failures) break;
        }
        while (!running.empty() || a.queued() > 0) {   // drain
            if (!running.empty()) {
                a.finish(running.begin()->second);
                running.erase(running.begin());
            }
            for (auto& it : a.admit()) {
                running[it.id] = it.bytes;
                ++admitted[it.id];
            }
            if (running.empty() && a.queued() > 0) {
                CHECK(false);   // something queued that can never be admitted
                break;
            }
        }
        CHECK(admitted.size() == next - 1);
        for (auto& kv : admitted) CHECK(kv.second == 1);
        CHECK(a.max_reserved() <= budget && a.max_active_seen() <= max_active);
    }
    if (failures) return 1;
    std::printf("admission: all checks passed\n");
    return 0;
}
