// std::stable_sort on one host thread: a second CPU reference beside the
// oracle for bench.py's CPU baseline (test and baseline infrastructure only;
// the library never loads it).
#include <algorithm>
#include <cstdint>

extern "C" int ref_stable_sort_u32(uint32_t* a, uint64_t n) {
    std::stable_sort(a, a + n);
    return 0;
}

extern "C" int ref_stable_sort_u64(uint64_t* a, uint64_t n) {
    std::stable_sort(a, a + n);
    return 0;
}
