// arena.h -- first-fit allocator of byte ranges inside one region of fixed
// capacity.  The serving loop holds its HBM budget as one device allocation
// and hands out ranges of it with this class, so admission by budget is an
// allocation that either succeeds or waits.  Host-only and free of CUDA, so
// its invariants can be checked by a plain C++ test.
#pragma once

#include <cstddef>
#include <iterator>
#include <map>

namespace priest {

class Arena {
public:
    explicit Arena(size_t capacity = 0, size_t align = 256) { reset(capacity, align); }

    // Forgets every range; the whole capacity (rounded down to the
    // alignment) becomes one free range.
    void reset(size_t capacity, size_t align)
    {
        align_ = align ? align : 1;
        cap_ = capacity / align_ * align_;
        free_.clear();
        if (cap_) free_[0] = cap_;
        used_ = peak_ = 0;
    }

    size_t round(size_t bytes) const { return (bytes + align_ - 1) / align_ * align_; }

    // First free range (lowest offset) that holds `bytes` rounded up to the
    // alignment.  Returns false, changing nothing, when none does.
    bool alloc(size_t bytes, size_t *off)
    {
        const size_t need = round(bytes ? bytes : 1);
        for (auto it = free_.begin(); it != free_.end(); ++it) {
            if (it->second < need) continue;
            const size_t at = it->first, len = it->second;
            free_.erase(it);
            if (len > need) free_[at + need] = len - need;
            used_ += need;
            if (used_ > peak_) peak_ = used_;
            *off = at;
            return true;
        }
        return false;
    }

    // Returns the range [off, off + bytes) given by alloc(bytes); neighbouring
    // free ranges are merged.
    void release(size_t off, size_t bytes)
    {
        size_t at = off, len = round(bytes ? bytes : 1);
        used_ -= len;
        auto next = free_.lower_bound(at);
        if (next != free_.begin()) {
            auto prev = std::prev(next);
            if (prev->first + prev->second == at) {
                at = prev->first;
                len += prev->second;
                free_.erase(prev);
            }
        }
        next = free_.lower_bound(at);
        if (next != free_.end() && at + len == next->first) {
            len += next->second;
            free_.erase(next);
        }
        free_[at] = len;
    }

    size_t capacity() const { return cap_; }
    size_t used() const { return used_; }
    size_t peak() const { return peak_; }
    size_t free_ranges() const { return free_.size(); }

    size_t largest_free() const
    {
        size_t m = 0;
        for (const auto &kv : free_)
            if (kv.second > m) m = kv.second;
        return m;
    }

    // Free ranges sorted, aligned, disjoint, not adjacent (fully merged),
    // inside the capacity, and summing with the used bytes to the capacity.
    bool check() const
    {
        size_t end = 0, total = 0;
        bool first = true;
        for (const auto &kv : free_) {
            if (kv.second == 0 || kv.first % align_ || kv.second % align_) return false;
            if (!first && kv.first <= end) return false;  // overlap or adjacency
            end = kv.first + kv.second;
            if (end > cap_) return false;
            total += kv.second;
            first = false;
        }
        return total + used_ == cap_;
    }

private:
    std::map<size_t, size_t> free_;  // offset -> length
    size_t cap_ = 0, align_ = 256, used_ = 0, peak_ = 0;
};

}  // namespace priest
