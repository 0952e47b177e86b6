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

# (S, OMAX) pairs used by the FP32 kernel shapes; L = S + OMAX + 1 rounded up
# to 4 samples.
SHAPES = [(20, 36), (20, 16), (28, 16), (20, 24), (12, 52), (28, 4)]
# (S, OMAX) pairs of the 16-bit kernel shapes; L = S + OMAX + 1 rounded up to
# 8 samples, held two per 32-bit register.
SHAPES16 = [(24, 40), (24, 24), (8, 60), (24, 32), (24, 8)]


def window(S, OMAX, q=4):
    return (S + OMAX + 1 + q - 1) // q * q


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


def emit16(S, OMAX, kind):
    """acc[s] += sample o + s of the packed window w (two samples per b32,
    low half first), with the mixed-precision add of the sample format."""
    L = window(S, OMAX, 8)
    LR = L // 2
    idx = S
    w0 = S + 1
    op = "add.rn.f32.f16" if kind == 0 else "add.rn.f32.bf16"
    lines = []
    lines.append(f"template <>\n__device__ __forceinline__ void add_shifted_h<{S}, {LR}, {OMAX}, {kind}>(int o, float (&acc)[{S}], const unsigned (&w)[{LR}]) {{")
    body = ["{"]
    body.append(".reg .b16 lo<" + str(LR) + ">, hi<" + str(LR) + ">;")
    body.append("tbl: .branchtargets " + ", ".join(f"C{o}" for o in range(OMAX + 1)) + ";")
    body.append(f"brx.idx.uni %{idx}, tbl;")
    for o in range(OMAX + 1):
        body.append(f"C{o}:")
        regs = sorted({(o + s) >> 1 for s in range(S)})
        for r in regs:
            body.append(f"mov.b32 {{lo{r}, hi{r}}}, %{w0 + r};")
        for s in range(S):
            i = o + s
            h = f"lo{i >> 1}" if i % 2 == 0 else f"hi{i >> 1}"
            body.append(f"{op} %{s}, {h}, %{s};")
        if o != OMAX:
            body.append("bra.uni CEND;")
    body.append("CEND:")
    body.append("}")
    asm = "\\n\"\n      \"".join(body)
    outs = ", ".join(f'"+f"(acc[{s}])' for s in range(S))
    ins = ", ".join([f'"r"(o)'] + [f'"r"(w[{i}])' for i in range(LR)])
    lines.append(f'  asm volatile(\n      "{asm}\\n"\n      : {outs}\n      : {ins});')
    lines.append("}\n")
    return "\n".join(lines)


# (S, OMAX) pairs of the FP32 DM-pair shapes (ALGO 2).
PAIRS = [(25, 11), (21, 15), (29, 11)]


def emit_pair(S, OMAX):
    """Two consecutive DM trials whose delays in a channel differ by d in
    [0, OMAX]: loads the S + d staged samples at lane 0's offset for the first
    trial (plus the lane's own offset, folded into the address), then
    a0[s] += w[s] and a1[s] += w[s + d].  One indexed branch per call."""
    lines = []
    lines.append(f"template <>\n__device__ __forceinline__ void add_pair<{S}, {OMAX}>(int d, unsigned addr, float (&a0)[{S}], float (&a1)[{S}]) {{")
    body = ["{"]
    body.append(f".reg .f32 w<{S + OMAX}>;")
    body.append("tbl: .branchtargets " + ", ".join(f"C{d}" for d in range(OMAX + 1)) + ";")
    ia = 2 * S
    idx = 2 * S + 1
    body.append(f"brx.idx.uni %{idx}, tbl;")
    for d in range(OMAX + 1):
        body.append(f"C{d}:")
        for k in range(S + d):
            body.append(f"ld.shared.f32 w{k}, [%{ia}+{4 * k}];")
        for s_ in range(S):
            body.append(f"add.f32 %{s_}, %{s_}, w{s_};")
            body.append(f"add.f32 %{S + s_}, %{S + s_}, w{s_ + d};")
        if d != OMAX:
            body.append("bra.uni CEND;")
    body.append("CEND:")
    body.append("}")
    asm = "\\n\"\n      \"".join(body)
    outs = ", ".join([f'"+f"(a0[{s_}])' for s_ in range(S)] + [f'"+f"(a1[{s_}])' for s_ in range(S)])
    ins = f'"r"(addr), "r"(d)'
    lines.append(f'  asm volatile(\n      "{asm}\\n"\n      : {outs}\n      : {ins}\n      : "memory");')
    lines.append("}\n")
    return "\n".join(lines)


# (S, OMAX) of the 16-bit DM-pair shapes (ALGO 2): S = 2 mod 4 so that lanes
# start an odd number of words apart.
PAIRS16 = [(26, 11), (22, 11)]


def emit_pair16(S, OMAX, kind):
    """16-bit version of emit_pair: samples two per 32-bit word (low half
    first); block index r (OMAX + 1) + d, with r the first trial's half-word
    offset inside its first word."""
    op = "add.rn.f32.f16" if kind == 0 else "add.rn.f32.bf16"
    nwmax = (1 + OMAX + S + 1) // 2
    lines = []
    lines.append(f"template <>\n__device__ __forceinline__ void add_pair16<{S}, {OMAX}, {kind}>(int b, unsigned addr, float (&a0)[{S}], float (&a1)[{S}]) {{")
    body = ["{"]
    body.append(f".reg .b32 w<{nwmax}>;")
    body.append(f".reg .b16 lo<{nwmax}>, hi<{nwmax}>;")
    nb = 2 * (OMAX + 1)
    body.append("tbl: .branchtargets " + ", ".join(f"C{b}" for b in range(nb)) + ";")
    ia = 2 * S
    idx = 2 * S + 1
    body.append(f"brx.idx.uni %{idx}, tbl;")
    for b in range(nb):
        r, d = b // (OMAX + 1), b % (OMAX + 1)
        nw = (r + d + S + 1) // 2
        body.append(f"C{b}:")
        for k in range(nw):
            body.append(f"ld.shared.b32 w{k}, [%{ia}+{4 * k}];")
        for k in range(nw):
            body.append(f"mov.b32 {{lo{k}, hi{k}}}, w{k};")
        def half(h):
            return f"lo{h >> 1}" if h % 2 == 0 else f"hi{h >> 1}"
        for s_ in range(S):
            body.append(f"{op} %{s_}, {half(r + s_)}, %{s_};")
            body.append(f"{op} %{S + s_}, {half(r + d + s_)}, %{S + s_};")
        if b != nb - 1:
            body.append("bra.uni CEND;")
    body.append("CEND:")
    body.append("}")
    asm = "\\n\"\n      \"".join(body)
    outs = ", ".join([f'"+f"(a0[{s_}])' for s_ in range(S)] + [f'"+f"(a1[{s_}])' for s_ in range(S)])
    ins = f'"r"(addr), "r"(b)'
    lines.append(f'  asm volatile(\n      "{asm}\\n"\n      : {outs}\n      : {ins}\n      : "memory");')
    lines.append("}\n")
    return "\n".join(lines)


# (S, MMAX) of the FP32 DM-quad shapes (ALGO 3): S odd (lanes start an odd
# number of words apart), consecutive-trial delay steps m or m + 1, m <= MMAX.
QUADS = [(25, 9), (31, 9), (23, 9), (41, 9)]


def quad_steps(b):
    """Block index b = m * 8 + bits -> offsets (0, o1, o2, o3) of the four
    trials: o_j - o_{j-1} = m + bit j-1 of `bits`."""
    m, bits = b // 8, b % 8
    o = [0]
    for j in range(3):
        o.append(o[-1] + m + ((bits >> j) & 1))
    return o


def emit_quad(S, MMAX):
    """Four consecutive DM trials sharing one window: loads the S + o3 staged
    samples from lane 0's offset for the first trial (plus the lane's own
    offset, folded into the address) and adds a_j[s] += w[s + o_j].  One
    indexed branch per call; the window is loaded in order and each sample is
    added into every trial that uses it, so only a few window registers are
    live at a time."""
    nb = 8 * (MMAX + 1)
    lines = []
    lines.append(f"template <>\n__device__ __forceinline__ void add_quad<{S}, {MMAX}>(int b, unsigned addr, float (&a)[4][{S}]) {{")
    body = ["{"]
    body.append(f".reg .f32 w<{S + 3 * (MMAX + 1)}>;")
    body.append("tbl: .branchtargets " + ", ".join(f"C{b}" for b in range(nb)) + ";")
    ia = 4 * S
    idx = 4 * S + 1
    body.append(f"brx.idx.uni %{idx}, tbl;")
    for b in range(nb):
        o = quad_steps(b)
        body.append(f"C{b}:")
        for k in range(S + o[3]):
            body.append(f"ld.shared.f32 w{k}, [%{ia}+{4 * k}];")
            for j in range(4):
                s_ = k - o[j]
                if 0 <= s_ < S:
                    r = j * S + s_
                    body.append(f"add.f32 %{r}, %{r}, w{k};")
        if b != nb - 1:
            body.append("bra.uni CEND;")
    body.append("CEND:")
    body.append("}")
    asm = "\\n\"\n      \"".join(body)
    outs = ", ".join(f'"+f"(a[{j}][{s_}])' for j in range(4) for s_ in range(S))
    ins = f'"r"(addr), "r"(b)'
    lines.append(f'  asm volatile(\n      "{asm}\\n"\n      : {outs}\n      : {ins}\n      : "memory");')
    lines.append("}\n")
    return "\n".join(lines)


# (S, MMAX) of the FP32 two-segment DM-quad shapes (ALGO 4): S odd.
QUADS2 = [(15, 9), (21, 9), (23, 9), (19, 9)]


def emit_quad2(S, MMAX):
    """emit_quad for two output segments 32 S samples apart: the lane's
    outputs s of segment 0 and of segment 1 share one 64-bit accumulator
    (segment 0 in the low word), and each window sample of the two segments
    (the second segment's window 128 S bytes after the first's) is packed
    into one register pair, so a single add.rn.f32x2 adds both; each lane's
    result is the same binary32 add as the scalar form."""
    nb = 8 * (MMAX + 1)
    nw = S + 3 * (MMAX + 1)
    ia = 4 * S
    body = ["{", f".reg .f32 u<{nw}>, v<{nw}>;", f".reg .b64 w<{nw}>;",
            "tbl: .branchtargets " + ", ".join(f"C{b}" for b in range(nb)) + ";",
            f"brx.idx.uni %{4 * S + 1}, tbl;"]
    for b in range(nb):
        o = quad_steps(b)
        body.append(f"C{b}:")
        for k in range(S + o[3]):
            body.append(f"ld.shared.f32 u{k}, [%{ia}+{4 * k}];")
            body.append(f"ld.shared.f32 v{k}, [%{ia}+{4 * k + 128 * S}];")
            body.append(f"mov.b64 w{k}, {{u{k}, v{k}}};")
            for j in range(4):
                s_ = k - o[j]
                if 0 <= s_ < S:
                    r = j * S + s_
                    body.append(f"add.rn.f32x2 %{r}, %{r}, w{k};")
        if b != nb - 1:
            body.append("bra.uni CEND;")
    body += ["CEND:", "}"]
    outs = ", ".join(f'"+l"(a[{j}][{s_}])' for j in range(4) for s_ in range(S))
    return _asm_fn(f"void add_quad2<{S}, {MMAX}>(int b, unsigned addr, unsigned long long (&a)[4][{S}])", body,
                   outs, '"r"(addr), "r"(b)')


# (S, MMAX) of the FP32 in-lane paired DM-quad shapes (ALGO 5): S odd.
QUADSP = [(45, 9), (43, 9), (27, 9), (25, 9), (29, 9)]


def emit_quadp(S, MMAX):
    """emit_quad with the lane's outputs s and s + H paired (H = S // 2):
    a[j][s] holds outputs s (low word) and s + H (high word) of trial j for
    s < H, t[j] its output 2 H.  The window w[0 .. S + o3) is loaded once, in
    order; pair k = (w[k], w[k + H]) is formed as soon as w[k + H] is loaded
    and added into a[j][k - o_j] of every trial j with 0 <= k - o_j < H by
    one add.rn.f32x2 (samples w[H .. H + o3) sit in two pairs; the assembler
    copies them).  Each lane's result is the same binary32 add as the
    scalar form."""
    H = S // 2
    nb = 8 * (MMAX + 1)
    nw = S + 3 * (MMAX + 1)
    ia = 4 * H + 4
    body = ["{", f".reg .f32 w<{nw}>;", f".reg .b64 p<{nw}>;",
            "tbl: .branchtargets " + ", ".join(f"C{b}" for b in range(nb)) + ";",
            f"brx.idx.uni %{ia + 1}, tbl;"]
    for b in range(nb):
        o = quad_steps(b)
        body.append(f"C{b}:")
        for i in range(S + o[3]):
            body.append(f"ld.shared.f32 w{i}, [%{ia}+{4 * i}];")
            k = i - H
            if k >= 0:
                used = [j for j in range(4) if 0 <= k - o[j] < H]
                if used:
                    body.append(f"mov.b64 p{k}, {{w{k}, w{i}}};")
                    for j in used:
                        r = j * H + (k - o[j])
                        body.append(f"add.rn.f32x2 %{r}, %{r}, p{k};")
            for j in range(4):
                if i - o[j] == 2 * H:
                    body.append(f"add.rn.f32 %{4 * H + j}, %{4 * H + j}, w{i};")
        if b != nb - 1:
            body.append("bra.uni CEND;")
    body += ["CEND:", "}"]
    outs = ", ".join([f'"+l"(a[{j}][{s_}])' for j in range(4) for s_ in range(H)] +
                     [f'"+f"(t[{j}])' for j in range(4)])
    return _asm_fn(f"void add_quadp<{S}, {MMAX}>(int b, unsigned addr, unsigned long long (&a)[4][{H}], "
                   f"float (&t)[4])", body, outs, '"r"(addr), "r"(b)')


# (S, MMAX) of the 16-bit float DM-quad shapes: S = 2 mod 4.
QUADS16 = [(26, 9), (30, 9)]
# (S, MMAX) of the 8-bit DM-quad shapes: S = 2 mod 4.
QUADS8 = [(26, 16), (22, 16), (18, 16), (30, 16), (14, 16)]


def _asm_fn(signature, body, outs, ins):
    asm = "\\n\"\n      \"".join(body)
    return (f"template <>\n__device__ __forceinline__ {signature} {{\n"
            f'  asm volatile(\n      "{asm}\\n"\n      : {outs}\n      : {ins}\n      : "memory");\n}}\n')


def emit_quad16(S, MMAX, kind):
    """16-bit float version of emit_quad: samples two per 32-bit word (low
    half first); block index (r (MMAX + 1) + m) 8 + bits, r = the first
    trial's half-word offset inside its first word."""
    op = "add.rn.f32.f16" if kind == 0 else "add.rn.f32.bf16"
    nwmax = (1 + 3 * (MMAX + 1) + S + 1) // 2
    nb = 2 * 8 * (MMAX + 1)
    body = ["{", f".reg .b32 w<{nwmax}>;", f".reg .b16 lo<{nwmax}>, hi<{nwmax}>;",
            "tbl: .branchtargets " + ", ".join(f"C{b}" for b in range(nb)) + ";",
            f"brx.idx.uni %{4 * S + 1}, tbl;"]
    for b in range(nb):
        r, mb = b // (8 * (MMAX + 1)), b % (8 * (MMAX + 1))
        p = [r + o for o in quad_steps(mb)]
        nw = (p[3] + S - 1) // 2 + 1
        body.append(f"C{b}:")
        for k in range(nw):
            body.append(f"ld.shared.b32 w{k}, [%{4 * S}+{4 * k}];")
            body.append(f"mov.b32 {{lo{k}, hi{k}}}, w{k};")
            for h in (2 * k, 2 * k + 1):
                for j in range(4):
                    s_ = h - p[j]
                    if 0 <= s_ < S:
                        half = f"lo{k}" if h % 2 == 0 else f"hi{k}"
                        body.append(f"{op} %{j * S + s_}, {half}, %{j * S + s_};")
        if b != nb - 1:
            body.append("bra.uni CEND;")
    body += ["CEND:", "}"]
    outs = ", ".join(f'"+f"(a[{j}][{s_}])' for j in range(4) for s_ in range(S))
    return _asm_fn(f"void add_quad16<{S}, {MMAX}, {kind}>(int b, unsigned addr, float (&a)[4][{S}])", body, outs,
                   '"r"(addr), "r"(b)')


def emit_quad8(S, MMAX):
    """8-bit samples staged as 16-bit integers, two per word.  Four trials
    share one window; block index (r (MMAX + 1) + m) 8 + bits as in
    emit_quad16.  Trial j's first sample sits p_j = r + o_j half-words into
    the window.  Even p_j: word p_j / 2 + i holds its outputs (2i, 2i + 1)
    and goes into e[j][i]; odd p_j: word (p_j - 1) / 2 + i holds its outputs
    (2i - 1, 2i) and goes into f[j][i] (i = 0 .. S / 2; the outputs -1 and S
    are never read).  Each add sums two 16-bit lanes; no lane carries into
    the next while at most 256 channels are summed."""
    H = S // 2
    nb = 2 * 8 * (MMAX + 1)
    nwmax = (1 + 3 * (MMAX + 1) + S + 1) // 2 + 1
    ne = 4 * H
    body = ["{", f".reg .b32 w<{nwmax}>;",
            "tbl: .branchtargets " + ", ".join(f"C{b}" for b in range(nb)) + ";",
            f"brx.idx.uni %{ne + 4 * (H + 1) + 1}, tbl;"]
    ia = ne + 4 * (H + 1)
    for b in range(nb):
        r, mb = b // (8 * (MMAX + 1)), b % (8 * (MMAX + 1))
        p = [r + o for o in quad_steps(mb)]
        uses = {}
        for j in range(4):
            if p[j] % 2 == 0:
                for i in range(H):
                    uses.setdefault(p[j] // 2 + i, []).append(j * H + i)
            else:
                for i in range(H + 1):
                    uses.setdefault((p[j] - 1) // 2 + i, []).append(ne + j * (H + 1) + i)
        body.append(f"C{b}:")
        for k in range(max(uses) + 1):
            body.append(f"ld.shared.b32 w{k}, [%{ia}+{4 * k}];")
            for op_ in uses.get(k, []):
                body.append(f"add.u32 %{op_}, %{op_}, w{k};")
        if b != nb - 1:
            body.append("bra.uni CEND;")
    body += ["CEND:", "}"]
    outs = ", ".join([f'"+r"(e[{j}][{i}])' for j in range(4) for i in range(H)] +
                     [f'"+r"(f[{j}][{i}])' for j in range(4) for i in range(H + 1)])
    return _asm_fn(f"void add_quad8<{S}, {MMAX}>(int b, unsigned addr, unsigned (&e)[4][{H}], "
                   f"unsigned (&f)[4][{H + 1}])", body, outs, '"r"(addr), "r"(b)')


# (S, MMAX, NCONS, variant) of the 8-bit DM-quad shapes whose stage loop runs
# inside the assembly (ALGO 9-11: variants 3, 4, 5).
QUADS8T = [(30, 16, 8, 3), (26, 16, 8, 3), (22, 16, 8, 3), (30, 16, 8, 4), (30, 16, 8, 5), (14, 16, 8, 4)]


def emit_quad8t(S, MMAX, NCONS, V=0):
    """emit_quad8 over every channel of a pipeline stage in one call, with
    threaded dispatch: the channel's block starts by fetching the next
    channel's (window offset, block index) pair from the stage's info (NCONS
    int4 apart per channel), issues every window load, then the adds (in
    load order, alternately as a 32-bit integer add and as a two-lane 16-bit
    add so that they spread over two execution pipes; both sum the two
    16-bit lanes exactly while no lane exceeds 16 bits), and ends with the
    indexed branch of the next channel instead of a jump back to a loop.
    Operands: e, f as in emit_quad8; then the lane's shared-memory base, the
    address of the stage's first info entry for this warp, and the number
    of channels in the stage (>= 1)."""
    # variant: 0 threaded, loads first, alternating add forms; 1 threaded,
    # loads first, 32-bit adds only; 2 threaded, loads and adds interleaved,
    # 32-bit adds only; 3 a loop around one dispatch, loads first,
    # alternating add forms; 4 the loop, interleaved, alternating forms; 5 the
    # loop, interleaved, 32-bit adds only
    threaded = V in (0, 1, 2)
    first = V in (0, 1, 3)
    alt = V in (0, 3, 4)
    H = S // 2
    nb = 2 * 8 * (MMAX + 1)
    nwmax = (1 + 3 * (MMAX + 1) + S + 1) // 2 + 1
    ne = 4 * H + 4 * (H + 1)
    sb, inf, nc = ne, ne + 1, ne + 2
    stride = 16 * NCONS
    body = ["{", ".reg .pred p;", f".reg .b32 w<{nwmax}>, ci, ip, ix, iy, ad;",
            "tbl: .branchtargets " + ", ".join(f"C{b}" for b in range(nb)) + ";",
            f"mov.u32 ip, %{inf};",
            "ld.shared.v2.u32 {ix, iy}, [ip];",
            "mov.u32 ci, 1;",
            f"add.u32 ad, %{sb}, ix;"]
    if threaded:
        body.append("brx.idx.uni iy, tbl;")
    else:
        body += ["LOOP:", "setp.lt.u32 p, ci, %{};".format(nc), "brx.idx.uni iy, tbl;"]
    for b in range(nb):
        r, mb = b // (8 * (MMAX + 1)), b % (8 * (MMAX + 1))
        p = [r + o for o in quad_steps(mb)]
        uses = {}
        for j in range(4):
            if p[j] % 2 == 0:
                for i in range(H):
                    uses.setdefault(p[j] // 2 + i, []).append(j * H + i)
            else:
                for i in range(H + 1):
                    uses.setdefault((p[j] - 1) // 2 + i, []).append(4 * H + j * (H + 1) + i)
        body.append(f"C{b}:")
        if threaded:
            body.append(f"setp.lt.u32 p, ci, %{nc};")
        body.append(f"@p add.u32 ip, ip, {stride};")
        body.append("ld.shared.v2.u32 {ix, iy}, [ip];")
        nw = max(uses) + 1
        n = 0
        if first:
            for k in range(nw):
                body.append(f"ld.shared.b32 w{k}, [ad+{4 * k}];")
        for k in range(nw):
            if not first:
                body.append(f"ld.shared.b32 w{k}, [ad+{4 * k}];")
            for op_ in uses.get(k, []):
                form = "add.u16x2" if alt and n % 2 else "add.u32"
                body.append(f"{form} %{op_}, %{op_}, w{k};")
                n += 1
        body.append("@!p bra.uni CEND;")
        body.append("add.u32 ci, ci, 1;")
        body.append(f"add.u32 ad, %{sb}, ix;")
        body.append("brx.idx.uni iy, tbl;" if threaded else "bra.uni LOOP;")
    body += ["CEND:", "}"]
    outs = ", ".join([f'"+r"(e[{j}][{i}])' for j in range(4) for i in range(H)] +
                     [f'"+r"(f[{j}][{i}])' for j in range(4) for i in range(H + 1)])
    return _asm_fn(f"void add_quad8t<{S}, {MMAX}, {NCONS}, {V}>(unsigned sbase, unsigned info, int nc, "
                   f"unsigned (&e)[4][{H}], unsigned (&f)[4][{H + 1}])", body, outs,
                   '"r"(sbase), "r"(info), "r"(nc)')


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
        "// two consecutive DM trials from one window of staged FP32 samples",
        "template <int S, int OMAX>",
        "__device__ __forceinline__ void add_pair(int d, unsigned addr, float (&a0)[S], float (&a1)[S]);",
        "",
        "// four consecutive DM trials from one window of staged FP32 samples;",
        "// block index = m * 8 + bits (trial j's offset exceeds trial j - 1's by",
        "// m + bit j - 1)",
        "template <int S, int MMAX>",
        "__device__ __forceinline__ void add_quad(int b, unsigned addr, float (&a)[4][S]);",
        "",
        "// four trials and two output segments 32 S samples apart, FP32 samples;",
        "// a[j][s] holds output s of both segments (segment 0 in the low word)",
        "template <int S, int MMAX>",
        "__device__ __forceinline__ void add_quad2(int b, unsigned addr, unsigned long long (&a)[4][S]);",
        "",
        "// four trials, FP32 samples, the lane's outputs s and s + S / 2 paired in",
        "// a[j][s] (low word first), output 2 (S / 2) in t[j]",
        "template <int S, int MMAX>",
        "__device__ __forceinline__ void add_quadp(int b, unsigned addr, unsigned long long (&a)[4][S / 2],",
        "                                          float (&t)[4]);",
        "",
        "// four trials, 16-bit float samples (kind 0 = binary16, 1 = bfloat16);",
        "// block index = (r * (MMAX + 1) + m) * 8 + bits, r = the first trial's",
        "// half-word offset in its first word",
        "template <int S, int MMAX, int KIND>",
        "__device__ __forceinline__ void add_quad16(int b, unsigned addr, float (&a)[4][S]);",
        "",
        "// four trials, 8-bit samples widened to 16-bit integers: e holds output",
        "// pairs (2i, 2i + 1), f output pairs (2i - 1, 2i), two 16-bit lanes a word",
        "template <int S, int MMAX>",
        "__device__ __forceinline__ void add_quad8(int b, unsigned addr, unsigned (&e)[4][S / 2],",
        "                                          unsigned (&f)[4][S / 2 + 1]);",
        "",
        "// every channel of a stage (emit_quad8t): the channel loop over the",
        "// stage's info entries inside the assembly",
        "template <int S, int MMAX, int NCONS, int V>",
        "__device__ __forceinline__ void add_quad8t(unsigned sbase, unsigned info, int nc,",
        "                                           unsigned (&e)[4][S / 2], unsigned (&f)[4][S / 2 + 1]);",
        "",
        "// the same for 16-bit samples (kind 0 = binary16, 1 = bfloat16), block",
        "// index = first trial's half-word offset r * (OMAX + 1) + d",
        "template <int S, int OMAX, int KIND>",
        "__device__ __forceinline__ void add_pair16(int b, unsigned addr, float (&a0)[S], float (&a1)[S]);",
        "",
        "// 16-bit samples, two per register; kind 0 = binary16, 1 = bfloat16.",
        "template <int S, int LR, int OMAX, int KIND>",
        "__device__ __forceinline__ void add_shifted_h(int o, float (&acc)[S], const unsigned (&w)[LR]);",
        "",
    ]
    for S, OMAX in SHAPES:
        out.append(emit(S, OMAX))
    for S, OMAX in SHAPES16:
        for kind in (0, 1):
            out.append(emit16(S, OMAX, kind))
    for S, OMAX in PAIRS:
        out.append(emit_pair(S, OMAX))
    for S, OMAX in PAIRS16:
        for kind in (0, 1):
            out.append(emit_pair16(S, OMAX, kind))
    for S, MMAX in QUADS:
        out.append(emit_quad(S, MMAX))
    for S, MMAX in QUADS2:
        out.append(emit_quad2(S, MMAX))
    for S, MMAX in QUADSP:
        out.append(emit_quadp(S, MMAX))
    for S, MMAX in QUADS16:
        for kind in (0, 1):
            out.append(emit_quad16(S, MMAX, kind))
    for S, MMAX in QUADS8:
        out.append(emit_quad8(S, MMAX))
    for S, MMAX, NCONS, V in QUADS8T:
        out.append(emit_quad8t(S, MMAX, NCONS, V))
    out.append("}  // namespace tp")
    with open(os.path.join(here, "dispatch_gen.cuh"), "w") as f:
        f.write("\n".join(out) + "\n")


if __name__ == "__main__":
    main()
