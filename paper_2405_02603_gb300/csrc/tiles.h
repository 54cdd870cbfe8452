// tiles.h -- radix schedule and tile shape of the generic line-transform
// engine, shared by every host file that launches it (the plan-based solve,
// the batched form, the no-allocation solve), so they cannot drift apart.
#pragma once
#include <cstring>

#include "fft_engine.cuh"

namespace fsp {

inline bool is_235_smooth(long long n) {
    if (n < 1) return false;
    for (int p : {2, 3, 5})
        while (n % p == 0) n /= p;
    return n == 1;
}

// Radix schedule: 5s, then 3s, then 8s, then one 4 or 2.
inline bool make_stages(int n, Stages &st) {
    std::memset(&st, 0, sizeof(st));
    st.n = n;
    int m = n;
    while (m % 5 == 0) m /= 5, ++st.n5;
    while (m % 3 == 0) m /= 3, ++st.n3;
    while (m % 8 == 0) m /= 8, ++st.n8;
    if (m % 4 == 0) m /= 4, st.last = 4;
    else if (m % 2 == 0) m /= 2, st.last = 2;
    return m == 1;
}

// Smallest threads-per-line (>= n/16) for which every stage keeps at most
// kMaxV complex values per thread.
inline int threads_per_line(const Stages &st) {
    const int radices[4] = {st.n5 ? 5 : 0, st.n3 ? 3 : 0, st.n8 ? 8 : 0, st.last};
    int tpl = st.n / 16;
    if (tpl < 1) tpl = 1;
    for (;; ++tpl) {
        bool ok = true;
        for (int R : radices) {
            if (!R) continue;
            const int nb = st.n / R;
            const int K = (nb + tpl - 1) / tpl;
            if (K > kMaxV / R) ok = false;
        }
        if (ok) return tpl;
    }
}

// Lines per CTA (2^lgL): as many as wanted, within 512 threads and 200 KB of
// shared memory (positions x (L+1) complex elements).
inline bool choose_tile(int positions, int tpl, size_t csize, int want_lgL, int &lgL) {
    for (lgL = want_lgL; lgL >= 0; --lgL) {
        const int L = 1 << lgL;
        const size_t sm = (size_t)positions * (L + 1) * csize;
        if (L * tpl <= 512 && sm <= 200 * 1024) return true;
    }
    return false;
}

struct TileCfg {
    Stages st;
    int tpl = 0, lgL = 0;
};

inline bool make_cfg(int n, int positions, size_t csize, int want_lgL, TileCfg &c) {
    if (!make_stages(n, c.st)) return false;
    c.tpl = threads_per_line(c.st);
    return choose_tile(positions, c.tpl, csize, want_lgL, c.lgL);
}

}  // namespace fsp
