// GENERATED by gen_chains.py -- do not edit by hand.
// Multi-word carry chains, each one inline-PTX statement (see gen_chains.py).
#pragma once

#include <cstdint>

namespace montgb {

template <int S> __device__ void mac_row(uint32_t (&t)[S], uint32_t& h0, uint32_t& h1,
                                         const uint32_t (&a)[S], uint32_t b);
template <int S> __device__ uint32_t sub_rows(uint32_t (&d)[S], const uint32_t (&t)[S],
                                            const uint32_t (&n)[S]);
template <int S> __device__ uint32_t add_word(uint32_t (&t)[S], uint32_t w);
template <int S> __device__ uint32_t sub_word(uint32_t (&t)[S], uint32_t w);
template <int S> __device__ uint32_t add_rows(uint32_t (&t)[S], const uint32_t (&u)[S]);

template <> __device__ __forceinline__ void mac_row<1>(uint32_t (&t)[1], uint32_t& h0, uint32_t& h1,
    const uint32_t (&a)[1], uint32_t b) {
  asm("mad.lo.cc.u32 %0, %3, %4, %0;\n\taddc.cc.u32 %1, %1, 0;\n\taddc.u32 %2, %2, 0;\n\tmad.hi.cc.u32 %1, %3, %4, %1;\n\taddc.u32 %2, %2, 0;"
      : "+r"(t[0]), "+r"(h0), "+r"(h1)
      : "r"(a[0]), "r"(b));
}

template <> __device__ __forceinline__ uint32_t sub_rows<1>(uint32_t (&d)[1], const uint32_t (&t)[1],
    const uint32_t (&n)[1]) {
  uint32_t bw;
  asm("sub.cc.u32 %0, %2, %3;\n\tsubc.u32 %1, 0, 0;"
      : "=r"(d[0]), "=r"(bw)
      : "r"(t[0]), "r"(n[0]));
  return bw & 1u;
}

template <> __device__ __forceinline__ uint32_t add_word<1>(uint32_t (&t)[1], uint32_t w) {
  uint32_t c;
  asm("add.cc.u32 %0, %0, %2;\n\taddc.u32 %1, 0, 0;"
      : "+r"(t[0]), "=r"(c)
      : "r"(w));
  return c & 1u;
}

template <> __device__ __forceinline__ uint32_t sub_word<1>(uint32_t (&t)[1], uint32_t w) {
  uint32_t c;
  asm("sub.cc.u32 %0, %0, %2;\n\tsubc.u32 %1, 0, 0;"
      : "+r"(t[0]), "=r"(c)
      : "r"(w));
  return c & 1u;
}

template <> __device__ __forceinline__ uint32_t add_rows<1>(uint32_t (&t)[1], const uint32_t (&u)[1]) {
  uint32_t c;
  asm("add.cc.u32 %0, %0, %2;\n\taddc.u32 %1, 0, 0;"
      : "+r"(t[0]), "=r"(c)
      : "r"(u[0]));
  return c & 1u;
}

template <> __device__ __forceinline__ void mac_row<2>(uint32_t (&t)[2], uint32_t& h0, uint32_t& h1,
    const uint32_t (&a)[2], uint32_t b) {
  asm("mad.lo.cc.u32 %0, %4, %6, %0;\n\tmadc.lo.cc.u32 %1, %5, %6, %1;\n\taddc.cc.u32 %2, %2, 0;\n\taddc.u32 %3, %3, 0;\n\tmad.hi.cc.u32 %1, %4, %6, %1;\n\tmadc.hi.cc.u32 %2, %5, %6, %2;\n\taddc.u32 %3, %3, 0;"
      : "+r"(t[0]), "+r"(t[1]), "+r"(h0), "+r"(h1)
      : "r"(a[0]), "r"(a[1]), "r"(b));
}

template <> __device__ __forceinline__ uint32_t sub_rows<2>(uint32_t (&d)[2], const uint32_t (&t)[2],
    const uint32_t (&n)[2]) {
  uint32_t bw;
  asm("sub.cc.u32 %0, %3, %5;\n\tsubc.cc.u32 %1, %4, %6;\n\tsubc.u32 %2, 0, 0;"
      : "=r"(d[0]), "=r"(d[1]), "=r"(bw)
      : "r"(t[0]), "r"(t[1]), "r"(n[0]), "r"(n[1]));
  return bw & 1u;
}

template <> __device__ __forceinline__ uint32_t add_word<2>(uint32_t (&t)[2], uint32_t w) {
  uint32_t c;
  asm("add.cc.u32 %0, %0, %3;\n\taddc.cc.u32 %1, %1, 0;\n\taddc.u32 %2, 0, 0;"
      : "+r"(t[0]), "+r"(t[1]), "=r"(c)
      : "r"(w));
  return c & 1u;
}

template <> __device__ __forceinline__ uint32_t sub_word<2>(uint32_t (&t)[2], uint32_t w) {
  uint32_t c;
  asm("sub.cc.u32 %0, %0, %3;\n\tsubc.cc.u32 %1, %1, 0;\n\tsubc.u32 %2, 0, 0;"
      : "+r"(t[0]), "+r"(t[1]), "=r"(c)
      : "r"(w));
  return c & 1u;
}

template <> __device__ __forceinline__ uint32_t add_rows<2>(uint32_t (&t)[2], const uint32_t (&u)[2]) {
  uint32_t c;
  asm("add.cc.u32 %0, %0, %3;\n\taddc.cc.u32 %1, %1, %4;\n\taddc.u32 %2, 0, 0;"
      : "+r"(t[0]), "+r"(t[1]), "=r"(c)
      : "r"(u[0]), "r"(u[1]));
  return c & 1u;
}

template <> __device__ __forceinline__ void mac_row<3>(uint32_t (&t)[3], uint32_t& h0, uint32_t& h1,
    const uint32_t (&a)[3], uint32_t b) {
  asm("mad.lo.cc.u32 %0, %5, %8, %0;\n\tmadc.lo.cc.u32 %1, %6, %8, %1;\n\tmadc.lo.cc.u32 %2, %7, %8, %2;\n\taddc.cc.u32 %3, %3, 0;\n\taddc.u32 %4, %4, 0;\n\tmad.hi.cc.u32 %1, %5, %8, %1;\n\tmadc.hi.cc.u32 %2, %6, %8, %2;\n\tmadc.hi.cc.u32 %3, %7, %8, %3;\n\taddc.u32 %4, %4, 0;"
      : "+r"(t[0]), "+r"(t[1]), "+r"(t[2]), "+r"(h0), "+r"(h1)
      : "r"(a[0]), "r"(a[1]), "r"(a[2]), "r"(b));
}

template <> __device__ __forceinline__ uint32_t sub_rows<3>(uint32_t (&d)[3], const uint32_t (&t)[3],
    const uint32_t (&n)[3]) {
  uint32_t bw;
  asm("sub.cc.u32 %0, %4, %7;\n\tsubc.cc.u32 %1, %5, %8;\n\tsubc.cc.u32 %2, %6, %9;\n\tsubc.u32 %3, 0, 0;"
      : "=r"(d[0]), "=r"(d[1]), "=r"(d[2]), "=r"(bw)
      : "r"(t[0]), "r"(t[1]), "r"(t[2]), "r"(n[0]), "r"(n[1]), "r"(n[2]));
  return bw & 1u;
}

template <> __device__ __forceinline__ uint32_t add_word<3>(uint32_t (&t)[3], uint32_t w) {
  uint32_t c;
  asm("add.cc.u32 %0, %0, %4;\n\taddc.cc.u32 %1, %1, 0;\n\taddc.cc.u32 %2, %2, 0;\n\taddc.u32 %3, 0, 0;"
      : "+r"(t[0]), "+r"(t[1]), "+r"(t[2]), "=r"(c)
      : "r"(w));
  return c & 1u;
}

template <> __device__ __forceinline__ uint32_t sub_word<3>(uint32_t (&t)[3], uint32_t w) {
  uint32_t c;
  asm("sub.cc.u32 %0, %0, %4;\n\tsubc.cc.u32 %1, %1, 0;\n\tsubc.cc.u32 %2, %2, 0;\n\tsubc.u32 %3, 0, 0;"
      : "+r"(t[0]), "+r"(t[1]), "+r"(t[2]), "=r"(c)
      : "r"(w));
  return c & 1u;
}

template <> __device__ __forceinline__ uint32_t add_rows<3>(uint32_t (&t)[3], const uint32_t (&u)[3]) {
  uint32_t c;
  asm("add.cc.u32 %0, %0, %4;\n\taddc.cc.u32 %1, %1, %5;\n\taddc.cc.u32 %2, %2, %6;\n\taddc.u32 %3, 0, 0;"
      : "+r"(t[0]), "+r"(t[1]), "+r"(t[2]), "=r"(c)
      : "r"(u[0]), "r"(u[1]), "r"(u[2]));
  return c & 1u;
}

template <> __device__ __forceinline__ void mac_row<4>(uint32_t (&t)[4], uint32_t& h0, uint32_t& h1,
    const uint32_t (&a)[4], uint32_t b) {
  asm("mad.lo.cc.u32 %0, %6, %10, %0;\n\tmadc.lo.cc.u32 %1, %7, %10, %1;\n\tmadc.lo.cc.u32 %2, %8, %10, %2;\n\tmadc.lo.cc.u32 %3, %9, %10, %3;\n\taddc.cc.u32 %4, %4, 0;\n\taddc.u32 %5, %5, 0;\n\tmad.hi.cc.u32 %1, %6, %10, %1;\n\tmadc.hi.cc.u32 %2, %7, %10, %2;\n\tmadc.hi.cc.u32 %3, %8, %10, %3;\n\tmadc.hi.cc.u32 %4, %9, %10, %4;\n\taddc.u32 %5, %5, 0;"
      : "+r"(t[0]), "+r"(t[1]), "+r"(t[2]), "+r"(t[3]), "+r"(h0), "+r"(h1)
      : "r"(a[0]), "r"(a[1]), "r"(a[2]), "r"(a[3]), "r"(b));
}

template <> __device__ __forceinline__ uint32_t sub_rows<4>(uint32_t (&d)[4], const uint32_t (&t)[4],
    const uint32_t (&n)[4]) {
  uint32_t bw;
  asm("sub.cc.u32 %0, %5, %9;\n\tsubc.cc.u32 %1, %6, %10;\n\tsubc.cc.u32 %2, %7, %11;\n\tsubc.cc.u32 %3, %8, %12;\n\tsubc.u32 %4, 0, 0;"
      : "=r"(d[0]), "=r"(d[1]), "=r"(d[2]), "=r"(d[3]), "=r"(bw)
      : "r"(t[0]), "r"(t[1]), "r"(t[2]), "r"(t[3]), "r"(n[0]), "r"(n[1]), "r"(n[2]), "r"(n[3]));
  return bw & 1u;
}

template <> __device__ __forceinline__ uint32_t add_word<4>(uint32_t (&t)[4], uint32_t w) {
  uint32_t c;
  asm("add.cc.u32 %0, %0, %5;\n\taddc.cc.u32 %1, %1, 0;\n\taddc.cc.u32 %2, %2, 0;\n\taddc.cc.u32 %3, %3, 0;\n\taddc.u32 %4, 0, 0;"
      : "+r"(t[0]), "+r"(t[1]), "+r"(t[2]), "+r"(t[3]), "=r"(c)
      : "r"(w));
  return c & 1u;
}

template <> __device__ __forceinline__ uint32_t sub_word<4>(uint32_t (&t)[4], uint32_t w) {
  uint32_t c;
  asm("sub.cc.u32 %0, %0, %5;\n\tsubc.cc.u32 %1, %1, 0;\n\tsubc.cc.u32 %2, %2, 0;\n\tsubc.cc.u32 %3, %3, 0;\n\tsubc.u32 %4, 0, 0;"
      : "+r"(t[0]), "+r"(t[1]), "+r"(t[2]), "+r"(t[3]), "=r"(c)
      : "r"(w));
  return c & 1u;
}

template <> __device__ __forceinline__ uint32_t add_rows<4>(uint32_t (&t)[4], const uint32_t (&u)[4]) {
  uint32_t c;
  asm("add.cc.u32 %0, %0, %5;\n\taddc.cc.u32 %1, %1, %6;\n\taddc.cc.u32 %2, %2, %7;\n\taddc.cc.u32 %3, %3, %8;\n\taddc.u32 %4, 0, 0;"
      : "+r"(t[0]), "+r"(t[1]), "+r"(t[2]), "+r"(t[3]), "=r"(c)
      : "r"(u[0]), "r"(u[1]), "r"(u[2]), "r"(u[3]));
  return c & 1u;
}

template <> __device__ __forceinline__ void mac_row<6>(uint32_t (&t)[6], uint32_t& h0, uint32_t& h1,
    const uint32_t (&a)[6], uint32_t b) {
  asm("mad.lo.cc.u32 %0, %8, %14, %0;\n\tmadc.lo.cc.u32 %1, %9, %14, %1;\n\tmadc.lo.cc.u32 %2, %10, %14, %2;\n\tmadc.lo.cc.u32 %3, %11, %14, %3;\n\tmadc.lo.cc.u32 %4, %12, %14, %4;\n\tmadc.lo.cc.u32 %5, %13, %14, %5;\n\taddc.cc.u32 %6, %6, 0;\n\taddc.u32 %7, %7, 0;\n\tmad.hi.cc.u32 %1, %8, %14, %1;\n\tmadc.hi.cc.u32 %2, %9, %14, %2;\n\tmadc.hi.cc.u32 %3, %10, %14, %3;\n\tmadc.hi.cc.u32 %4, %11, %14, %4;\n\tmadc.hi.cc.u32 %5, %12, %14, %5;\n\tmadc.hi.cc.u32 %6, %13, %14, %6;\n\taddc.u32 %7, %7, 0;"
      : "+r"(t[0]), "+r"(t[1]), "+r"(t[2]), "+r"(t[3]), "+r"(t[4]), "+r"(t[5]), "+r"(h0), "+r"(h1)
      : "r"(a[0]), "r"(a[1]), "r"(a[2]), "r"(a[3]), "r"(a[4]), "r"(a[5]), "r"(b));
}

template <> __device__ __forceinline__ uint32_t sub_rows<6>(uint32_t (&d)[6], const uint32_t (&t)[6],
    const uint32_t (&n)[6]) {
  uint32_t bw;
  asm("sub.cc.u32 %0, %7, %13;\n\tsubc.cc.u32 %1, %8, %14;\n\tsubc.cc.u32 %2, %9, %15;\n\tsubc.cc.u32 %3, %10, %16;\n\tsubc.cc.u32 %4, %11, %17;\n\tsubc.cc.u32 %5, %12, %18;\n\tsubc.u32 %6, 0, 0;"
      : "=r"(d[0]), "=r"(d[1]), "=r"(d[2]), "=r"(d[3]), "=r"(d[4]), "=r"(d[5]), "=r"(bw)
      : "r"(t[0]), "r"(t[1]), "r"(t[2]), "r"(t[3]), "r"(t[4]), "r"(t[5]), "r"(n[0]), "r"(n[1]), "r"(n[2]), "r"(n[3]), "r"(n[4]), "r"(n[5]));
  return bw & 1u;
}

template <> __device__ __forceinline__ uint32_t add_word<6>(uint32_t (&t)[6], uint32_t w) {
  uint32_t c;
  asm("add.cc.u32 %0, %0, %7;\n\taddc.cc.u32 %1, %1, 0;\n\taddc.cc.u32 %2, %2, 0;\n\taddc.cc.u32 %3, %3, 0;\n\taddc.cc.u32 %4, %4, 0;\n\taddc.cc.u32 %5, %5, 0;\n\taddc.u32 %6, 0, 0;"
      : "+r"(t[0]), "+r"(t[1]), "+r"(t[2]), "+r"(t[3]), "+r"(t[4]), "+r"(t[5]), "=r"(c)
      : "r"(w));
  return c & 1u;
}

template <> __device__ __forceinline__ uint32_t sub_word<6>(uint32_t (&t)[6], uint32_t w) {
  uint32_t c;
  asm("sub.cc.u32 %0, %0, %7;\n\tsubc.cc.u32 %1, %1, 0;\n\tsubc.cc.u32 %2, %2, 0;\n\tsubc.cc.u32 %3, %3, 0;\n\tsubc.cc.u32 %4, %4, 0;\n\tsubc.cc.u32 %5, %5, 0;\n\tsubc.u32 %6, 0, 0;"
      : "+r"(t[0]), "+r"(t[1]), "+r"(t[2]), "+r"(t[3]), "+r"(t[4]), "+r"(t[5]), "=r"(c)
      : "r"(w));
  return c & 1u;
}

template <> __device__ __forceinline__ uint32_t add_rows<6>(uint32_t (&t)[6], const uint32_t (&u)[6]) {
  uint32_t c;
  asm("add.cc.u32 %0, %0, %7;\n\taddc.cc.u32 %1, %1, %8;\n\taddc.cc.u32 %2, %2, %9;\n\taddc.cc.u32 %3, %3, %10;\n\taddc.cc.u32 %4, %4, %11;\n\taddc.cc.u32 %5, %5, %12;\n\taddc.u32 %6, 0, 0;"
      : "+r"(t[0]), "+r"(t[1]), "+r"(t[2]), "+r"(t[3]), "+r"(t[4]), "+r"(t[5]), "=r"(c)
      : "r"(u[0]), "r"(u[1]), "r"(u[2]), "r"(u[3]), "r"(u[4]), "r"(u[5]));
  return c & 1u;
}

template <> __device__ __forceinline__ void mac_row<8>(uint32_t (&t)[8], uint32_t& h0, uint32_t& h1,
    const uint32_t (&a)[8], uint32_t b) {
  asm("mad.lo.cc.u32 %0, %10, %18, %0;\n\tmadc.lo.cc.u32 %1, %11, %18, %1;\n\tmadc.lo.cc.u32 %2, %12, %18, %2;\n\tmadc.lo.cc.u32 %3, %13, %18, %3;\n\tmadc.lo.cc.u32 %4, %14, %18, %4;\n\tmadc.lo.cc.u32 %5, %15, %18, %5;\n\tmadc.lo.cc.u32 %6, %16, %18, %6;\n\tmadc.lo.cc.u32 %7, %17, %18, %7;\n\taddc.cc.u32 %8, %8, 0;\n\taddc.u32 %9, %9, 0;\n\tmad.hi.cc.u32 %1, %10, %18, %1;\n\tmadc.hi.cc.u32 %2, %11, %18, %2;\n\tmadc.hi.cc.u32 %3, %12, %18, %3;\n\tmadc.hi.cc.u32 %4, %13, %18, %4;\n\tmadc.hi.cc.u32 %5, %14, %18, %5;\n\tmadc.hi.cc.u32 %6, %15, %18, %6;\n\tmadc.hi.cc.u32 %7, %16, %18, %7;\n\tmadc.hi.cc.u32 %8, %17, %18, %8;\n\taddc.u32 %9, %9, 0;"
      : "+r"(t[0]), "+r"(t[1]), "+r"(t[2]), "+r"(t[3]), "+r"(t[4]), "+r"(t[5]), "+r"(t[6]), "+r"(t[7]), "+r"(h0), "+r"(h1)
      : "r"(a[0]), "r"(a[1]), "r"(a[2]), "r"(a[3]), "r"(a[4]), "r"(a[5]), "r"(a[6]), "r"(a[7]), "r"(b));
}

template <> __device__ __forceinline__ uint32_t sub_rows<8>(uint32_t (&d)[8], const uint32_t (&t)[8],
    const uint32_t (&n)[8]) {
  uint32_t bw;
  asm("sub.cc.u32 %0, %9, %17;\n\tsubc.cc.u32 %1, %10, %18;\n\tsubc.cc.u32 %2, %11, %19;\n\tsubc.cc.u32 %3, %12, %20;\n\tsubc.cc.u32 %4, %13, %21;\n\tsubc.cc.u32 %5, %14, %22;\n\tsubc.cc.u32 %6, %15, %23;\n\tsubc.cc.u32 %7, %16, %24;\n\tsubc.u32 %8, 0, 0;"
      : "=r"(d[0]), "=r"(d[1]), "=r"(d[2]), "=r"(d[3]), "=r"(d[4]), "=r"(d[5]), "=r"(d[6]), "=r"(d[7]), "=r"(bw)
      : "r"(t[0]), "r"(t[1]), "r"(t[2]), "r"(t[3]), "r"(t[4]), "r"(t[5]), "r"(t[6]), "r"(t[7]), "r"(n[0]), "r"(n[1]), "r"(n[2]), "r"(n[3]), "r"(n[4]), "r"(n[5]), "r"(n[6]), "r"(n[7]));
  return bw & 1u;
}

template <> __device__ __forceinline__ uint32_t add_word<8>(uint32_t (&t)[8], uint32_t w) {
  uint32_t c;
  asm("add.cc.u32 %0, %0, %9;\n\taddc.cc.u32 %1, %1, 0;\n\taddc.cc.u32 %2, %2, 0;\n\taddc.cc.u32 %3, %3, 0;\n\taddc.cc.u32 %4, %4, 0;\n\taddc.cc.u32 %5, %5, 0;\n\taddc.cc.u32 %6, %6, 0;\n\taddc.cc.u32 %7, %7, 0;\n\taddc.u32 %8, 0, 0;"
      : "+r"(t[0]), "+r"(t[1]), "+r"(t[2]), "+r"(t[3]), "+r"(t[4]), "+r"(t[5]), "+r"(t[6]), "+r"(t[7]), "=r"(c)
      : "r"(w));
  return c & 1u;
}

template <> __device__ __forceinline__ uint32_t sub_word<8>(uint32_t (&t)[8], uint32_t w) {
  uint32_t c;
  asm("sub.cc.u32 %0, %0, %9;\n\tsubc.cc.u32 %1, %1, 0;\n\tsubc.cc.u32 %2, %2, 0;\n\tsubc.cc.u32 %3, %3, 0;\n\tsubc.cc.u32 %4, %4, 0;\n\tsubc.cc.u32 %5, %5, 0;\n\tsubc.cc.u32 %6, %6, 0;\n\tsubc.cc.u32 %7, %7, 0;\n\tsubc.u32 %8, 0, 0;"
      : "+r"(t[0]), "+r"(t[1]), "+r"(t[2]), "+r"(t[3]), "+r"(t[4]), "+r"(t[5]), "+r"(t[6]), "+r"(t[7]), "=r"(c)
      : "r"(w));
  return c & 1u;
}

template <> __device__ __forceinline__ uint32_t add_rows<8>(uint32_t (&t)[8], const uint32_t (&u)[8]) {
  uint32_t c;
  asm("add.cc.u32 %0, %0, %9;\n\taddc.cc.u32 %1, %1, %10;\n\taddc.cc.u32 %2, %2, %11;\n\taddc.cc.u32 %3, %3, %12;\n\taddc.cc.u32 %4, %4, %13;\n\taddc.cc.u32 %5, %5, %14;\n\taddc.cc.u32 %6, %6, %15;\n\taddc.cc.u32 %7, %7, %16;\n\taddc.u32 %8, 0, 0;"
      : "+r"(t[0]), "+r"(t[1]), "+r"(t[2]), "+r"(t[3]), "+r"(t[4]), "+r"(t[5]), "+r"(t[6]), "+r"(t[7]), "=r"(c)
      : "r"(u[0]), "r"(u[1]), "r"(u[2]), "r"(u[3]), "r"(u[4]), "r"(u[5]), "r"(u[6]), "r"(u[7]));
  return c & 1u;
}

template <> __device__ __forceinline__ void mac_row<12>(uint32_t (&t)[12], uint32_t& h0, uint32_t& h1,
    const uint32_t (&a)[12], uint32_t b) {
  asm("mad.lo.cc.u32 %0, %14, %26, %0;\n\tmadc.lo.cc.u32 %1, %15, %26, %1;\n\tmadc.lo.cc.u32 %2, %16, %26, %2;\n\tmadc.lo.cc.u32 %3, %17, %26, %3;\n\tmadc.lo.cc.u32 %4, %18, %26, %4;\n\tmadc.lo.cc.u32 %5, %19, %26, %5;\n\tmadc.lo.cc.u32 %6, %20, %26, %6;\n\tmadc.lo.cc.u32 %7, %21, %26, %7;\n\tmadc.lo.cc.u32 %8, %22, %26, %8;\n\tmadc.lo.cc.u32 %9, %23, %26, %9;\n\tmadc.lo.cc.u32 %10, %24, %26, %10;\n\tmadc.lo.cc.u32 %11, %25, %26, %11;\n\taddc.cc.u32 %12, %12, 0;\n\taddc.u32 %13, %13, 0;\n\tmad.hi.cc.u32 %1, %14, %26, %1;\n\tmadc.hi.cc.u32 %2, %15, %26, %2;\n\tmadc.hi.cc.u32 %3, %16, %26, %3;\n\tmadc.hi.cc.u32 %4, %17, %26, %4;\n\tmadc.hi.cc.u32 %5, %18, %26, %5;\n\tmadc.hi.cc.u32 %6, %19, %26, %6;\n\tmadc.hi.cc.u32 %7, %20, %26, %7;\n\tmadc.hi.cc.u32 %8, %21, %26, %8;\n\tmadc.hi.cc.u32 %9, %22, %26, %9;\n\tmadc.hi.cc.u32 %10, %23, %26, %10;\n\tmadc.hi.cc.u32 %11, %24, %26, %11;\n\tmadc.hi.cc.u32 %12, %25, %26, %12;\n\taddc.u32 %13, %13, 0;"
      : "+r"(t[0]), "+r"(t[1]), "+r"(t[2]), "+r"(t[3]), "+r"(t[4]), "+r"(t[5]), "+r"(t[6]), "+r"(t[7]), "+r"(t[8]), "+r"(t[9]), "+r"(t[10]), "+r"(t[11]), "+r"(h0), "+r"(h1)
      : "r"(a[0]), "r"(a[1]), "r"(a[2]), "r"(a[3]), "r"(a[4]), "r"(a[5]), "r"(a[6]), "r"(a[7]), "r"(a[8]), "r"(a[9]), "r"(a[10]), "r"(a[11]), "r"(b));
}

template <> __device__ __forceinline__ uint32_t sub_rows<12>(uint32_t (&d)[12], const uint32_t (&t)[12],
    const uint32_t (&n)[12]) {
  uint32_t bw;
  asm("sub.cc.u32 %0, %13, %25;\n\tsubc.cc.u32 %1, %14, %26;\n\tsubc.cc.u32 %2, %15, %27;\n\tsubc.cc.u32 %3, %16, %28;\n\tsubc.cc.u32 %4, %17, %29;\n\tsubc.cc.u32 %5, %18, %30;\n\tsubc.cc.u32 %6, %19, %31;\n\tsubc.cc.u32 %7, %20, %32;\n\tsubc.cc.u32 %8, %21, %33;\n\tsubc.cc.u32 %9, %22, %34;\n\tsubc.cc.u32 %10, %23, %35;\n\tsubc.cc.u32 %11, %24, %36;\n\tsubc.u32 %12, 0, 0;"
      : "=r"(d[0]), "=r"(d[1]), "=r"(d[2]), "=r"(d[3]), "=r"(d[4]), "=r"(d[5]), "=r"(d[6]), "=r"(d[7]), "=r"(d[8]), "=r"(d[9]), "=r"(d[10]), "=r"(d[11]), "=r"(bw)
      : "r"(t[0]), "r"(t[1]), "r"(t[2]), "r"(t[3]), "r"(t[4]), "r"(t[5]), "r"(t[6]), "r"(t[7]), "r"(t[8]), "r"(t[9]), "r"(t[10]), "r"(t[11]), "r"(n[0]), "r"(n[1]), "r"(n[2]), "r"(n[3]), "r"(n[4]), "r"(n[5]), "r"(n[6]), "r"(n[7]), "r"(n[8]), "r"(n[9]), "r"(n[10]), "r"(n[11]));
  return bw & 1u;
}

template <> __device__ __forceinline__ uint32_t add_word<12>(uint32_t (&t)[12], uint32_t w) {
  uint32_t c;
  asm("add.cc.u32 %0, %0, %13;\n\taddc.cc.u32 %1, %1, 0;\n\taddc.cc.u32 %2, %2, 0;\n\taddc.cc.u32 %3, %3, 0;\n\taddc.cc.u32 %4, %4, 0;\n\taddc.cc.u32 %5, %5, 0;\n\taddc.cc.u32 %6, %6, 0;\n\taddc.cc.u32 %7, %7, 0;\n\taddc.cc.u32 %8, %8, 0;\n\taddc.cc.u32 %9, %9, 0;\n\taddc.cc.u32 %10, %10, 0;\n\taddc.cc.u32 %11, %11, 0;\n\taddc.u32 %12, 0, 0;"
      : "+r"(t[0]), "+r"(t[1]), "+r"(t[2]), "+r"(t[3]), "+r"(t[4]), "+r"(t[5]), "+r"(t[6]), "+r"(t[7]), "+r"(t[8]), "+r"(t[9]), "+r"(t[10]), "+r"(t[11]), "=r"(c)
      : "r"(w));
  return c & 1u;
}

template <> __device__ __forceinline__ uint32_t sub_word<12>(uint32_t (&t)[12], uint32_t w) {
  uint32_t c;
  asm("sub.cc.u32 %0, %0, %13;\n\tsubc.cc.u32 %1, %1, 0;\n\tsubc.cc.u32 %2, %2, 0;\n\tsubc.cc.u32 %3, %3, 0;\n\tsubc.cc.u32 %4, %4, 0;\n\tsubc.cc.u32 %5, %5, 0;\n\tsubc.cc.u32 %6, %6, 0;\n\tsubc.cc.u32 %7, %7, 0;\n\tsubc.cc.u32 %8, %8, 0;\n\tsubc.cc.u32 %9, %9, 0;\n\tsubc.cc.u32 %10, %10, 0;\n\tsubc.cc.u32 %11, %11, 0;\n\tsubc.u32 %12, 0, 0;"
      : "+r"(t[0]), "+r"(t[1]), "+r"(t[2]), "+r"(t[3]), "+r"(t[4]), "+r"(t[5]), "+r"(t[6]), "+r"(t[7]), "+r"(t[8]), "+r"(t[9]), "+r"(t[10]), "+r"(t[11]), "=r"(c)
      : "r"(w));
  return c & 1u;
}

template <> __device__ __forceinline__ uint32_t add_rows<12>(uint32_t (&t)[12], const uint32_t (&u)[12]) {
  uint32_t c;
  asm("add.cc.u32 %0, %0, %13;\n\taddc.cc.u32 %1, %1, %14;\n\taddc.cc.u32 %2, %2, %15;\n\taddc.cc.u32 %3, %3, %16;\n\taddc.cc.u32 %4, %4, %17;\n\taddc.cc.u32 %5, %5, %18;\n\taddc.cc.u32 %6, %6, %19;\n\taddc.cc.u32 %7, %7, %20;\n\taddc.cc.u32 %8, %8, %21;\n\taddc.cc.u32 %9, %9, %22;\n\taddc.cc.u32 %10, %10, %23;\n\taddc.cc.u32 %11, %11, %24;\n\taddc.u32 %12, 0, 0;"
      : "+r"(t[0]), "+r"(t[1]), "+r"(t[2]), "+r"(t[3]), "+r"(t[4]), "+r"(t[5]), "+r"(t[6]), "+r"(t[7]), "+r"(t[8]), "+r"(t[9]), "+r"(t[10]), "+r"(t[11]), "=r"(c)
      : "r"(u[0]), "r"(u[1]), "r"(u[2]), "r"(u[3]), "r"(u[4]), "r"(u[5]), "r"(u[6]), "r"(u[7]), "r"(u[8]), "r"(u[9]), "r"(u[10]), "r"(u[11]));
  return c & 1u;
}

template <> __device__ __forceinline__ void mac_row<16>(uint32_t (&t)[16], uint32_t& h0, uint32_t& h1,
    const uint32_t (&a)[16], uint32_t b) {
  asm("mad.lo.cc.u32 %0, %18, %34, %0;\n\tmadc.lo.cc.u32 %1, %19, %34, %1;\n\tmadc.lo.cc.u32 %2, %20, %34, %2;\n\tmadc.lo.cc.u32 %3, %21, %34, %3;\n\tmadc.lo.cc.u32 %4, %22, %34, %4;\n\tmadc.lo.cc.u32 %5, %23, %34, %5;\n\tmadc.lo.cc.u32 %6, %24, %34, %6;\n\tmadc.lo.cc.u32 %7, %25, %34, %7;\n\tmadc.lo.cc.u32 %8, %26, %34, %8;\n\tmadc.lo.cc.u32 %9, %27, %34, %9;\n\tmadc.lo.cc.u32 %10, %28, %34, %10;\n\tmadc.lo.cc.u32 %11, %29, %34, %11;\n\tmadc.lo.cc.u32 %12, %30, %34, %12;\n\tmadc.lo.cc.u32 %13, %31, %34, %13;\n\tmadc.lo.cc.u32 %14, %32, %34, %14;\n\tmadc.lo.cc.u32 %15, %33, %34, %15;\n\taddc.cc.u32 %16, %16, 0;\n\taddc.u32 %17, %17, 0;\n\tmad.hi.cc.u32 %1, %18, %34, %1;\n\tmadc.hi.cc.u32 %2, %19, %34, %2;\n\tmadc.hi.cc.u32 %3, %20, %34, %3;\n\tmadc.hi.cc.u32 %4, %21, %34, %4;\n\tmadc.hi.cc.u32 %5, %22, %34, %5;\n\tmadc.hi.cc.u32 %6, %23, %34, %6;\n\tmadc.hi.cc.u32 %7, %24, %34, %7;\n\tmadc.hi.cc.u32 %8, %25, %34, %8;\n\tmadc.hi.cc.u32 %9, %26, %34, %9;\n\tmadc.hi.cc.u32 %10, %27, %34, %10;\n\tmadc.hi.cc.u32 %11, %28, %34, %11;\n\tmadc.hi.cc.u32 %12, %29, %34, %12;\n\tmadc.hi.cc.u32 %13, %30, %34, %13;\n\tmadc.hi.cc.u32 %14, %31, %34, %14;\n\tmadc.hi.cc.u32 %15, %32, %34, %15;\n\tmadc.hi.cc.u32 %16, %33, %34, %16;\n\taddc.u32 %17, %17, 0;"
      : "+r"(t[0]), "+r"(t[1]), "+r"(t[2]), "+r"(t[3]), "+r"(t[4]), "+r"(t[5]), "+r"(t[6]), "+r"(t[7]), "+r"(t[8]), "+r"(t[9]), "+r"(t[10]), "+r"(t[11]), "+r"(t[12]), "+r"(t[13]), "+r"(t[14]), "+r"(t[15]), "+r"(h0), "+r"(h1)
      : "r"(a[0]), "r"(a[1]), "r"(a[2]), "r"(a[3]), "r"(a[4]), "r"(a[5]), "r"(a[6]), "r"(a[7]), "r"(a[8]), "r"(a[9]), "r"(a[10]), "r"(a[11]), "r"(a[12]), "r"(a[13]), "r"(a[14]), "r"(a[15]), "r"(b));
}

template <> __device__ __forceinline__ uint32_t sub_rows<16>(uint32_t (&d)[16], const uint32_t (&t)[16],
    const uint32_t (&n)[16]) {
  uint32_t bw;
  asm("sub.cc.u32 %0, %17, %33;\n\tsubc.cc.u32 %1, %18, %34;\n\tsubc.cc.u32 %2, %19, %35;\n\tsubc.cc.u32 %3, %20, %36;\n\tsubc.cc.u32 %4, %21, %37;\n\tsubc.cc.u32 %5, %22, %38;\n\tsubc.cc.u32 %6, %23, %39;\n\tsubc.cc.u32 %7, %24, %40;\n\tsubc.cc.u32 %8, %25, %41;\n\tsubc.cc.u32 %9, %26, %42;\n\tsubc.cc.u32 %10, %27, %43;\n\tsubc.cc.u32 %11, %28, %44;\n\tsubc.cc.u32 %12, %29, %45;\n\tsubc.cc.u32 %13, %30, %46;\n\tsubc.cc.u32 %14, %31, %47;\n\tsubc.cc.u32 %15, %32, %48;\n\tsubc.u32 %16, 0, 0;"
      : "=r"(d[0]), "=r"(d[1]), "=r"(d[2]), "=r"(d[3]), "=r"(d[4]), "=r"(d[5]), "=r"(d[6]), "=r"(d[7]), "=r"(d[8]), "=r"(d[9]), "=r"(d[10]), "=r"(d[11]), "=r"(d[12]), "=r"(d[13]), "=r"(d[14]), "=r"(d[15]), "=r"(bw)
      : "r"(t[0]), "r"(t[1]), "r"(t[2]), "r"(t[3]), "r"(t[4]), "r"(t[5]), "r"(t[6]), "r"(t[7]), "r"(t[8]), "r"(t[9]), "r"(t[10]), "r"(t[11]), "r"(t[12]), "r"(t[13]), "r"(t[14]), "r"(t[15]), "r"(n[0]), "r"(n[1]), "r"(n[2]), "r"(n[3]), "r"(n[4]), "r"(n[5]), "r"(n[6]), "r"(n[7]), "r"(n[8]), "r"(n[9]), "r"(n[10]), "r"(n[11]), "r"(n[12]), "r"(n[13]), "r"(n[14]), "r"(n[15]));
  return bw & 1u;
}

template <> __device__ __forceinline__ uint32_t add_word<16>(uint32_t (&t)[16], uint32_t w) {
  uint32_t c;
  asm("add.cc.u32 %0, %0, %17;\n\taddc.cc.u32 %1, %1, 0;\n\taddc.cc.u32 %2, %2, 0;\n\taddc.cc.u32 %3, %3, 0;\n\taddc.cc.u32 %4, %4, 0;\n\taddc.cc.u32 %5, %5, 0;\n\taddc.cc.u32 %6, %6, 0;\n\taddc.cc.u32 %7, %7, 0;\n\taddc.cc.u32 %8, %8, 0;\n\taddc.cc.u32 %9, %9, 0;\n\taddc.cc.u32 %10, %10, 0;\n\taddc.cc.u32 %11, %11, 0;\n\taddc.cc.u32 %12, %12, 0;\n\taddc.cc.u32 %13, %13, 0;\n\taddc.cc.u32 %14, %14, 0;\n\taddc.cc.u32 %15, %15, 0;\n\taddc.u32 %16, 0, 0;"
      : "+r"(t[0]), "+r"(t[1]), "+r"(t[2]), "+r"(t[3]), "+r"(t[4]), "+r"(t[5]), "+r"(t[6]), "+r"(t[7]), "+r"(t[8]), "+r"(t[9]), "+r"(t[10]), "+r"(t[11]), "+r"(t[12]), "+r"(t[13]), "+r"(t[14]), "+r"(t[15]), "=r"(c)
      : "r"(w));
  return c & 1u;
}

template <> __device__ __forceinline__ uint32_t sub_word<16>(uint32_t (&t)[16], uint32_t w) {
  uint32_t c;
  asm("sub.cc.u32 %0, %0, %17;\n\tsubc.cc.u32 %1, %1, 0;\n\tsubc.cc.u32 %2, %2, 0;\n\tsubc.cc.u32 %3, %3, 0;\n\tsubc.cc.u32 %4, %4, 0;\n\tsubc.cc.u32 %5, %5, 0;\n\tsubc.cc.u32 %6, %6, 0;\n\tsubc.cc.u32 %7, %7, 0;\n\tsubc.cc.u32 %8, %8, 0;\n\tsubc.cc.u32 %9, %9, 0;\n\tsubc.cc.u32 %10, %10, 0;\n\tsubc.cc.u32 %11, %11, 0;\n\tsubc.cc.u32 %12, %12, 0;\n\tsubc.cc.u32 %13, %13, 0;\n\tsubc.cc.u32 %14, %14, 0;\n\tsubc.cc.u32 %15, %15, 0;\n\tsubc.u32 %16, 0, 0;"
      : "+r"(t[0]), "+r"(t[1]), "+r"(t[2]), "+r"(t[3]), "+r"(t[4]), "+r"(t[5]), "+r"(t[6]), "+r"(t[7]), "+r"(t[8]), "+r"(t[9]), "+r"(t[10]), "+r"(t[11]), "+r"(t[12]), "+r"(t[13]), "+r"(t[14]), "+r"(t[15]), "=r"(c)
      : "r"(w));
  return c & 1u;
}

template <> __device__ __forceinline__ uint32_t add_rows<16>(uint32_t (&t)[16], const uint32_t (&u)[16]) {
  uint32_t c;
  asm("add.cc.u32 %0, %0, %17;\n\taddc.cc.u32 %1, %1, %18;\n\taddc.cc.u32 %2, %2, %19;\n\taddc.cc.u32 %3, %3, %20;\n\taddc.cc.u32 %4, %4, %21;\n\taddc.cc.u32 %5, %5, %22;\n\taddc.cc.u32 %6, %6, %23;\n\taddc.cc.u32 %7, %7, %24;\n\taddc.cc.u32 %8, %8, %25;\n\taddc.cc.u32 %9, %9, %26;\n\taddc.cc.u32 %10, %10, %27;\n\taddc.cc.u32 %11, %11, %28;\n\taddc.cc.u32 %12, %12, %29;\n\taddc.cc.u32 %13, %13, %30;\n\taddc.cc.u32 %14, %14, %31;\n\taddc.cc.u32 %15, %15, %32;\n\taddc.u32 %16, 0, 0;"
      : "+r"(t[0]), "+r"(t[1]), "+r"(t[2]), "+r"(t[3]), "+r"(t[4]), "+r"(t[5]), "+r"(t[6]), "+r"(t[7]), "+r"(t[8]), "+r"(t[9]), "+r"(t[10]), "+r"(t[11]), "+r"(t[12]), "+r"(t[13]), "+r"(t[14]), "+r"(t[15]), "=r"(c)
      : "r"(u[0]), "r"(u[1]), "r"(u[2]), "r"(u[3]), "r"(u[4]), "r"(u[5]), "r"(u[6]), "r"(u[7]), "r"(u[8]), "r"(u[9]), "r"(u[10]), "r"(u[11]), "r"(u[12]), "r"(u[13]), "r"(u[14]), "r"(u[15]));
  return c & 1u;
}

}  // namespace montgb
