// Fixed-width types and a type selector for the kernels compiled at run time
// (NVRTC has no standard headers).
#pragma once

typedef unsigned char u8;
typedef unsigned short u16;
typedef unsigned int u32;
typedef unsigned long long u64;
typedef long long i64;

namespace mpm {

template <bool B, class X, class Y>
struct Cond {
    typedef X T;
};
template <class X, class Y>
struct Cond<false, X, Y> {
    typedef Y T;
};

}  // namespace mpm
