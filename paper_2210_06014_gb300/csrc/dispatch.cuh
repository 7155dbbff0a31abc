// dispatch.cuh -- maps runtime (R, J) to template instantiations.
// Supported: R in {4, 8, 16, 32}, J in {4, 8, 16, 32}, 4*J >= R.
#pragma once

#include <type_traits>

namespace sft {

template <int V>
using ic = std::integral_constant<int, V>;

template <int R, typename F>
inline void dispatch_j(int J, F &&f) {
    switch (J) {
        case 4:
            if constexpr (4 * 4 >= R) f(ic<R>{}, ic<4>{});
            break;
        case 8: f(ic<R>{}, ic<8>{}); break;
        case 16: f(ic<R>{}, ic<16>{}); break;
        case 32: f(ic<R>{}, ic<32>{}); break;
        default: break;
    }
}

template <typename F>
inline void dispatch_rj(int R, int J, F &&f) {
    switch (R) {
        case 4: dispatch_j<4>(J, f); break;
        case 8: dispatch_j<8>(J, f); break;
        case 16: dispatch_j<16>(J, f); break;
        case 32: dispatch_j<32>(J, f); break;
        default: break;
    }
}

template <typename F>
inline void dispatch_r(int R, F &&f) {
    switch (R) {
        case 4: f(ic<4>{}); break;
        case 8: f(ic<8>{}); break;
        case 16: f(ic<16>{}); break;
        case 32: f(ic<32>{}); break;
        default: break;
    }
}

}  // namespace sft

// BODY sees constexpr ints R_ and J_.
#define SFT_DISPATCH_RJ(R, J, BODY)                                              \
    ::sft::dispatch_rj((R), (J), [&](auto r_c, auto j_c) {                       \
        constexpr int R_ = decltype(r_c)::value;                                 \
        constexpr int J_ = decltype(j_c)::value;                                 \
        BODY;                                                                    \
    })

#define SFT_DISPATCH_R(R, BODY)                                                  \
    ::sft::dispatch_r((R), [&](auto r_c) {                                       \
        constexpr int R_ = decltype(r_c)::value;                                 \
        BODY;                                                                    \
    })
