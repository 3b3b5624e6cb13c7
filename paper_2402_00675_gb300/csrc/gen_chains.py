#!/usr/bin/env python3
"""Generate cios_chains.cuh: multi-word carry chains as single inline-PTX statements.

Each primitive is emitted as ONE asm statement so that nothing the compiler
schedules can sit between the instructions that set and consume the carry
flag.  Sizes S are the limbs a thread holds (thread-per-element CIOS uses
S = k; a team of L lanes per element uses S = k / L).

Primitives (all arrays little-endian 32-bit limbs):
  mac_row<S>(t, h0, h1, a, b)   (t, h0, h1) += a * b, where h0 and h1 are the
                                two words above t (positions S and S+1)
  sub_rows<S>(d, t, n)          d = t - n, returns the borrow out (0 or 1)
  add_word<S>(t, w)             t += w (w a 32-bit word), returns the carry out
  sub_word<S>(t, w)             t -= w, returns the borrow out
  add_rows<S>(t, u)             t += u, returns the carry out
Run: python gen_chains.py > cios_chains.cuh
"""

SIZES = (1, 2, 3, 4, 6, 8, 12, 16)


def mac_row(S):
    # operands: t[0..S-1] -> %0..%{S-1}, h0 %S, h1 %S+1, a[0..S-1] %S+2.., b last
    t = [f"%{i}" for i in range(S)]
    h0, h1 = f"%{S}", f"%{S + 1}"
    a = [f"%{S + 2 + i}" for i in range(S)]
    b = f"%{2 * S + 2}"
    body = []
    # low halves: t[j] += lo(a[j] b), carry into h0, h1
    body.append(f"mad.lo.cc.u32 {t[0]}, {a[0]}, {b}, {t[0]};")
    for j in range(1, S):
        body.append(f"madc.lo.cc.u32 {t[j]}, {a[j]}, {b}, {t[j]};")
    body.append(f"addc.cc.u32 {h0}, {h0}, 0;")
    body.append(f"addc.u32 {h1}, {h1}, 0;")
    # high halves: t[j+1] += hi(a[j] b) for j < S-1, h0 += hi(a[S-1] b), carry into h1
    dst = t[1:] + [h0]
    body.append(f"mad.hi.cc.u32 {dst[0]}, {a[0]}, {b}, {dst[0]};")
    for j in range(1, S):
        body.append(f"madc.hi.cc.u32 {dst[j]}, {a[j]}, {b}, {dst[j]};")
    body.append(f"addc.u32 {h1}, {h1}, 0;")
    outs = ", ".join([f'"+r"(t[{i}])' for i in range(S)] + ['"+r"(h0)', '"+r"(h1)'])
    ins = ", ".join([f'"r"(a[{i}])' for i in range(S)] + ['"r"(b)'])
    asm = "\\n\\t".join(body)
    return (f"template <> __device__ __forceinline__ void mac_row<{S}>(uint32_t (&t)[{S}], "
            f"uint32_t& h0, uint32_t& h1,\n    const uint32_t (&a)[{S}], uint32_t b) {{\n"
            f"  asm(\"{asm}\"\n      : {outs}\n      : {ins});\n}}\n")


def sub_rows(S):
    d = [f"%{i}" for i in range(S)]
    bw = f"%{S}"
    t = [f"%{S + 1 + i}" for i in range(S)]
    n = [f"%{2 * S + 1 + i}" for i in range(S)]
    body = [f"sub.cc.u32 {d[0]}, {t[0]}, {n[0]};"]
    for j in range(1, S):
        body.append(f"subc.cc.u32 {d[j]}, {t[j]}, {n[j]};")
    body.append(f"subc.u32 {bw}, 0, 0;")
    outs = ", ".join([f'"=r"(d[{i}])' for i in range(S)] + ['"=r"(bw)'])
    ins = ", ".join([f'"r"(t[{i}])' for i in range(S)] + [f'"r"(n[{i}])' for i in range(S)])
    asm = "\\n\\t".join(body)
    return (f"template <> __device__ __forceinline__ uint32_t sub_rows<{S}>(uint32_t (&d)[{S}], "
            f"const uint32_t (&t)[{S}],\n    const uint32_t (&n)[{S}]) {{\n  uint32_t bw;\n"
            f"  asm(\"{asm}\"\n      : {outs}\n      : {ins});\n  return bw & 1u;\n}}\n")


def add_word(S, op):
    t = [f"%{i}" for i in range(S)]
    c = f"%{S}"
    w = f"%{S + 1}"
    first, rest, fin = ("add.cc.u32", "addc.cc.u32", "addc.u32") if op == "add" else \
        ("sub.cc.u32", "subc.cc.u32", "subc.u32")
    body = [f"{first} {t[0]}, {t[0]}, {w};"]
    for j in range(1, S):
        body.append(f"{rest} {t[j]}, {t[j]}, 0;")
    body.append(f"{fin} {c}, 0, 0;")
    outs = ", ".join([f'"+r"(t[{i}])' for i in range(S)] + ['"=r"(c)'])
    asm = "\\n\\t".join(body)
    name = "add_word" if op == "add" else "sub_word"
    return (f"template <> __device__ __forceinline__ uint32_t {name}<{S}>(uint32_t (&t)[{S}], "
            f"uint32_t w) {{\n  uint32_t c;\n  asm(\"{asm}\"\n      : {outs}\n      : \"r\"(w));\n"
            f"  return c & 1u;\n}}\n")


def add_rows(S):
    t = [f"%{i}" for i in range(S)]
    c = f"%{S}"
    u = [f"%{S + 1 + i}" for i in range(S)]
    body = [f"add.cc.u32 {t[0]}, {t[0]}, {u[0]};"]
    for j in range(1, S):
        body.append(f"addc.cc.u32 {t[j]}, {t[j]}, {u[j]};")
    body.append(f"addc.u32 {c}, 0, 0;")
    outs = ", ".join([f'"+r"(t[{i}])' for i in range(S)] + ['"=r"(c)'])
    ins = ", ".join(f'"r"(u[{i}])' for i in range(S))
    asm = "\\n\\t".join(body)
    return (f"template <> __device__ __forceinline__ uint32_t add_rows<{S}>(uint32_t (&t)[{S}], "
            f"const uint32_t (&u)[{S}]) {{\n  uint32_t c;\n  asm(\"{asm}\"\n      : {outs}\n      : {ins});\n"
            f"  return c & 1u;\n}}\n")


def main():
    out = ["// GENERATED by gen_chains.py -- do not edit by hand.",
           "// Multi-word carry chains, each one inline-PTX statement (see gen_chains.py).",
           "#pragma once", "", "#include <cstdint>", "", "namespace montgb {", "",
           "template <int S> __device__ void mac_row(uint32_t (&t)[S], uint32_t& h0, uint32_t& h1,",
           "                                         const uint32_t (&a)[S], uint32_t b);",
           "template <int S> __device__ uint32_t sub_rows(uint32_t (&d)[S], const uint32_t (&t)[S],",
           "                                            const uint32_t (&n)[S]);",
           "template <int S> __device__ uint32_t add_word(uint32_t (&t)[S], uint32_t w);",
           "template <int S> __device__ uint32_t sub_word(uint32_t (&t)[S], uint32_t w);",
           "template <int S> __device__ uint32_t add_rows(uint32_t (&t)[S], const uint32_t (&u)[S]);",
           ""]
    for S in SIZES:
        out.append(mac_row(S))
        out.append(sub_rows(S))
        out.append(add_word(S, "add"))
        out.append(add_word(S, "sub"))
        out.append(add_rows(S))
    out.append("}  // namespace montgb")
    print("\n".join(out))


if __name__ == "__main__":
    main()
