"""Writes dispatch_gen.cuh: the shifted-add dispatch of the dedispersion kernel.

For each register shape (S outputs per lane, window of L registers, offsets
0..OMAX) it emits one inline-PTX function

    acc[s] += w[o + s]   for s < S,  o warp-uniform in [0, OMAX]

as an indexed branch (``brx.idx.uni`` over a ``.branchtargets`` table) into
OMAX + 1 straight-line blocks of S ``add.f32``.  A C++ ``switch`` over the same
cases compiles to a compare tree; the table keeps the dispatch to one branch.

Run from this directory: ``python gen_dispatch.py`` (the build step also runs
it when the header is older than this script).
"""
import os

# (S, OMAX) pairs used by the kernel shapes; L = S + OMAX + 1 rounded up to 4.
SHAPES = [(20, 36), (20, 16), (28, 16), (20, 24), (12, 52), (28, 4)]


def window(S, OMAX):
    return (S + OMAX + 1 + 3) // 4 * 4


def emit(S, OMAX):
    L = window(S, OMAX)
    idx = S  # operand number of the offset
    w0 = S + 1
    lines = []
    lines.append(f"template <>\n__device__ __forceinline__ void add_shifted<{S}, {L}, {OMAX}>(int o, float (&acc)[{S}], const float (&w)[{L}]) {{")
    body = ["{"]
    body.append("tbl: .branchtargets " + ", ".join(f"C{o}" for o in range(OMAX + 1)) + ";")
    body.append(f"brx.idx.uni %{idx}, tbl;")
    for o in range(OMAX + 1):
        body.append(f"C{o}:")
        for s in range(S):
            body.append(f"add.f32 %{s}, %{s}, %{w0 + o + s};")
        if o != OMAX:
            body.append("bra.uni CEND;")
    body.append("CEND:")
    body.append("}")
    asm = "\\n\"\n      \"".join(body)
    outs = ", ".join(f'"+f"(acc[{s}])' for s in range(S))
    ins = ", ".join([f'"r"(o)'] + [f'"f"(w[{i}])' for i in range(L)])
    lines.append(f'  asm volatile(\n      "{asm}\\n"\n      : {outs}\n      : {ins});')
    lines.append("}\n")
    return "\n".join(lines)


def main():
    here = os.path.dirname(os.path.abspath(__file__))
    out = [
        "// Generated by gen_dispatch.py -- do not edit.",
        "// acc[s] += w[o + s] (s < S) for a warp-uniform offset o in [0, OMAX],",
        "// as one indexed branch into straight-line add blocks.",
        "#pragma once",
        "",
        "namespace tp {",
        "",
        "template <int S, int L, int OMAX>",
        "__device__ __forceinline__ void add_shifted(int o, float (&acc)[S], const float (&w)[L]);",
        "",
    ]
    for S, OMAX in SHAPES:
        out.append(emit(S, OMAX))
    out.append("}  // namespace tp")
    with open(os.path.join(here, "dispatch_gen.cuh"), "w") as f:
        f.write("\n".join(out) + "\n")


if __name__ == "__main__":
    main()
