// Admission policy of the request server: which queued requests go on the device
// next, given a budget of device bytes and a number of slots.  Plain C++ (no CUDA),
// so that the policy can be checked on its own.
//
// Requests are considered in arrival order.  One that fits (a free slot, and its
// reserved bytes within what the admitted requests leave of the budget) is admitted.
// One that does not fit may be overtaken by later requests that do, but only
// max_bypass times: once its count is reached, nothing behind it is admitted until
// it has been, so a large request cannot be starved by a stream of small ones.
#pragma once

#include <cstddef>
#include <cstdint>
#include <deque>
#include <vector>

namespace mg {

class Admission {
public:
    struct Item {
        uint64_t id;
        size_t bytes;
        int bypassed;
    };

    Admission(size_t budget, int max_active, int max_bypass)
        : budget_(budget), max_active_(max_active), max_bypass_(max_bypass) {}

    // A request of this size can never be admitted.
    bool too_large(size_t bytes) const { return bytes > budget_; }

    void push(uint64_t id, size_t bytes) { queue_.push_back(Item{id, bytes, 0}); }
    // Put a request back at the head (re-admission after a refused allocation).
    void push_front(uint64_t id, size_t bytes) { queue_.push_front(Item{id, bytes, max_bypass_}); }

    // Remove a queued request; false if it is not queued.
    bool remove(uint64_t id) {
        for (auto it = queue_.begin(); it != queue_.end(); ++it)
            if (it->id == id) {
                queue_.erase(it);
                return true;
            }
        return false;
    }

    // Admit what fits now, in order; returns the admitted items.
    std::vector<Item> admit() {
        std::vector<Item> out;
        for (size_t i = 0; i < queue_.size() && active_ < max_active_;) {
            Item& it = queue_[i];
            if (it.bytes <= budget_ - reserved_) {
                out.push_back(it);
                reserved_ += it.bytes;
                ++active_;
                bool limit = false;   // an overtaken request reached its limit
                for (size_t j = 0; j < i; ++j) limit |= ++queue_[j].bypassed >= max_bypass_;
                queue_.erase(queue_.begin() + (long)i);
                if (active_ > max_active_seen_) max_active_seen_ = active_;
                if (reserved_ > max_reserved_) max_reserved_ = reserved_;
                if (limit) break;
                continue;
            }
            if (it.bypassed >= max_bypass_) break;   // it waits for no one else
            ++i;
        }
        return out;
    }

    // An admitted request of `bytes` reserved has finished.
    void finish(size_t bytes) {
        reserved_ -= bytes;
        --active_;
    }

    size_t budget() const { return budget_; }
    size_t reserved() const { return reserved_; }
    size_t max_reserved() const { return max_reserved_; }
    int active() const { return active_; }
    int max_active_seen() const { return max_active_seen_; }
    int queued() const { return (int)queue_.size(); }
    const std::deque<Item>& queue() const { return queue_; }

private:
    size_t budget_;
    int max_active_, max_bypass_;
    size_t reserved_ = 0, max_reserved_ = 0;
    int active_ = 0, max_active_seen_ = 0;
    std::deque<Item> queue_;
};

}  // namespace mg
