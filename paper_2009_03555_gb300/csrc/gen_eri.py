"""Generator of the per-angular-momentum-class ERI device code (run by the build).

For every canonical class (la lb | lc ld) of s/p/d shells (la >= lb, lc >= ld,
bra pair class >= ket pair class: 21 classes) it emits a traits struct with

  vrr<R>(G, geo, acc, comp)
                        Obara-Saika / Head-Gordon-Pople vertical recursion for
                        one primitive quartet: builds [e0|f0]^(0) for
                        |e| in [la, la+lb], |f| in [lc, lc+ld] from the
                        auxiliary integrals G_m = [00|00]^(m), m = 0..L, and
                        adds them into the contracted accumulators acc
                        (compensated summation with comp in FP32).
  hrr<R>(acc, AB, CD, out)
                        horizontal recursion on the contracted integrals,
                        (a,b+1_i| = (a+1_i,b| + AB_i (a,b|, first on the bra
                        then on the ket, giving (ab|cd) in Cartesian order.

Everything is straight-line code (one local per recursion node), so the
compiler keeps it in registers where it can.  The emitted flop counts (every
multiply and add as written) are exported per class for roofline accounting.

Recursions (Obara & Saika 1986; Head-Gordon & Pople 1988), with
PA = P - A, QC = Q - C, WP = W - P = -(rho/p) PQ, WQ = W - Q = (rho/q) PQ:
  [e+1_i|0]^(m) = PA_i [e|0]^(m) + WP_i [e|0]^(m+1)
                  + e_i/(2p) ([e-1_i|0]^(m) - rho/p [e-1_i|0]^(m+1))
  [e|f+1_i]^(m) = QC_i [e|f]^(m) + WQ_i [e|f]^(m+1)
                  + f_i/(2q) ([e|f-1_i]^(m) - rho/q [e|f-1_i]^(m+1))
                  + e_i/(2(p+q)) [e-1_i|f]^(m+1)
The same recursion holds for the erf/erfc-attenuated kernels once the G_m are
the attenuated auxiliary integrals.
"""
from __future__ import annotations

import os
import sys

LMAX = 2
PAIR_CLASSES = [(0, 0), (1, 0), (1, 1), (2, 0), (2, 1), (2, 2)]  # ss ps pp ds dp dd


def comps(l):
    out = []
    for lx in range(l, -1, -1):
        for ly in range(l - lx, -1, -1):
            out.append((lx, ly, l - lx - ly))
    return out


def comps_range(lo, hi):
    out = []
    for l in range(lo, hi + 1):
        out.extend(comps(l))
    return out


def quartet_classes():
    out = []
    for ib, (la, lb) in enumerate(PAIR_CLASSES):
        for ik, (lc, ld) in enumerate(PAIR_CLASSES):
            if ik <= ib:
                out.append((ib, ik, la, lb, lc, ld))
    return out


def _sub(v, i, k=1):
    w = list(v)
    w[i] -= k
    return tuple(w)


def _add(v, i, k=1):
    w = list(v)
    w[i] += k
    return tuple(w)


def _nm(v):
    return "".join(str(x) for x in v)


AX = "xyz"
# classes with more contracted accumulators than this get out-of-line
# recursion functions (their working set lives in local memory anyway)
INLINE_MAX_ACC = 160

# Blocks per SM the per-thread kernel of a class is compiled for (launch bound;
# 3 caps it at 168 registers).  Measured on GB300 (100-atom HSE cluster, mixed):
# three blocks are 17-20 % faster for (pp|ps), (ds|ds) and (dd|ss) and 3 % for
# (dp|ps) despite some spilling, but 43 % slower for (pp|pp) and 6 % for
# (ds|pp), which keep one.
PT_MIN_BLOCKS = {(1, 1, 1, 0): 3, (2, 0, 2, 0): 3, (2, 2, 0, 0): 3, (2, 1, 1, 0): 3}
# Per-thread classes whose primitive loop prefetches the next ket primitive
# pair (measured on GB300, 100-atom HSE build: 2-8 % faster for these, 3-15 %
# slower for the others, where the extra live pair costs registers).
PT_PREFETCH = {(0, 0, 0, 0), (1, 0, 1, 0), (1, 1, 0, 0), (1, 1, 1, 0), (2, 0, 0, 0), (2, 0, 1, 1), (2, 2, 0, 0)}
# Warp-split classes whose FP32 chunk accumulators live in shared memory
# (measured, 100-atom HSE build: (dp|pp) 3.8 % faster, spill-free at 153
# registers; (dd|dd) unchanged, (dp|dp) 3.5 % slower).
SPLIT_SMEM_ACC = {(2, 1, 1, 1)}
# FP32 warp-split classes with their own warps per lockstep block (absent:
# the kernel's rule by recursion size, 12 for the wide classes).  Measured on
# GB300, 100-atom HSE build, 16-warp blocks (128 registers) against the rule:
# (dp|pp) 347 -> 296 ms, (dp|ds) 278 -> 250, (dp|dp) 297 -> 273, (dd|ps)
# 132 -> 114, (dd|ds) 136 -> 122; (dd|pp) and (dd|dp) unchanged or slower.
SPLIT_WARPS = {(2, 1, 1, 1): 16, (2, 1, 2, 0): 16, (2, 1, 2, 1): 16, (2, 2, 1, 0): 16, (2, 2, 2, 0): 16}


class VRR:
    def __init__(self, la, lb, lc, ld):
        self.la, self.lb, self.lc, self.ld = la, lb, lc, ld
        self.L = la + lb + lc + ld
        self.E = comps_range(la, la + lb)
        self.F = comps_range(lc, lc + ld)
        self.names = {}
        self.lines = []
        self.flops = 0

    def node(self, e, f, m):
        key = (e, f, m)
        if key in self.names:
            return self.names[key]
        if sum(e) == 0 and sum(f) == 0:
            name = f"G[{m}]"
            self.names[key] = name
            return name
        terms = []
        fl = 0
        if sum(f) > 0:
            i = next(k for k in range(3) if f[k] > 0)
            f1 = _sub(f, i)
            terms.append(f"QC{AX[i]} * {self.node(e, f1, m)}")
            terms.append(f"WQ{AX[i]} * {self.node(e, f1, m + 1)}")
            fl += 2
            if f1[i] > 0:
                f2 = _sub(f1, i)
                a, b = self.node(e, f2, m), self.node(e, f2, m + 1)
                terms.append(f"R({f1[i]}) * oo2q * ({a} - roq * {b})")
                fl += 3 + (f1[i] > 1)
            if e[i] > 0:
                terms.append(f"R({e[i]}) * oo2pq * {self.node(_sub(e, i), f1, m + 1)}")
                fl += 1 + (e[i] > 1)
        else:
            i = next(k for k in range(3) if e[k] > 0)
            e1 = _sub(e, i)
            terms.append(f"PA{AX[i]} * {self.node(e1, f, m)}")
            terms.append(f"WP{AX[i]} * {self.node(e1, f, m + 1)}")
            fl += 2
            if e1[i] > 0:
                e2 = _sub(e1, i)
                a, b = self.node(e2, f, m), self.node(e2, f, m + 1)
                terms.append(f"R({e1[i]}) * oo2p * ({a} - rop * {b})")
                fl += 3 + (e1[i] > 1)
        fl += len(terms) - 1
        self.flops += fl
        name = f"v{_nm(e)}_{_nm(f)}_{m}"
        self.names[key] = name
        self.lines.append(f"    const R {name} = " + " + ".join(terms) + ";")
        return name

    def emit(self):
        acc_lines = []
        nf = len(self.F)
        for ie, e in enumerate(self.E):
            for jf, f in enumerate(self.F):
                nm = self.node(e, f, 0)
                acc_lines.append(f"    kacc<R>(acc[{ie * nf + jf}], comp[{ie * nf + jf}], {nm});")
                self.flops += 1
        return self.lines + acc_lines


class HRR:
    """Contracted horizontal recursion, bra then ket."""

    def __init__(self, la, lb, lc, ld):
        self.la, self.lb, self.lc, self.ld = la, lb, lc, ld
        self.E = comps_range(la, la + lb)
        self.F = comps_range(lc, lc + ld)
        self.eidx = {e: i for i, e in enumerate(self.E)}
        self.fidx = {f: i for i, f in enumerate(self.F)}
        self.lines = []
        self.flops = 0

    def emit(self):
        la, lb, lc, ld = self.la, self.lb, self.lc, self.ld
        nf = len(self.F)
        # bra: (a b | f] for every f
        bra = {}

        def bnode(a, b, jf):
            key = (a, b, jf)
            if key in bra:
                return bra[key]
            if sum(b) == 0:
                nm = f"acc[{self.eidx[a] * nf + jf}]"
            else:
                i = next(k for k in range(3) if b[k] > 0)
                b1 = _sub(b, i)
                x = bnode(_add(a, i), b1, jf)
                y = bnode(a, b1, jf)
                nm = f"h{_nm(a)}_{_nm(b)}_{jf}"
                self.lines.append(f"    const R {nm} = {x} + AB{AX[i]} * {y};")
                self.flops += 2
            bra[key] = nm
            return nm

        A, B, C, D = comps(la), comps(lb), comps(lc), comps(ld)
        ket = {}

        def knode(ia, ib, c, d):
            key = (ia, ib, c, d)
            if key in ket:
                return ket[key]
            if sum(d) == 0:
                nm = bnode(A[ia], B[ib], self.fidx[c])
            else:
                i = next(k for k in range(3) if d[k] > 0)
                d1 = _sub(d, i)
                x = knode(ia, ib, _add(c, i), d1)
                y = knode(ia, ib, c, d1)
                nm = f"k{ia}_{ib}_{_nm(c)}_{_nm(d)}"
                self.lines.append(f"    const R {nm} = {x} + CD{AX[i]} * {y};")
                self.flops += 2
            ket[key] = nm
            return nm

        nB, nC, nD = len(B), len(C), len(D)
        outs = []
        for ia in range(len(A)):
            for ib in range(nB):
                for ic, c in enumerate(C):
                    for id_, d in enumerate(D):
                        nm = knode(ia, ib, c, d)
                        outs.append(f"    out[{((ia * nB + ib) * nC + ic) * nD + id_}] = {nm};")
        return self.lines + outs


def gen_class(ib, ik, la, lb, lc, ld):
    v = VRR(la, lb, lc, ld)
    vl = v.emit()
    h = HRR(la, lb, lc, ld)
    hl = h.emit()
    name = f"Cls{la}{lb}{lc}{ld}"
    NA, NB, NC, ND = (len(comps(x)) for x in (la, lb, lc, ld))
    src = []
    nacc = len(v.E) * len(v.F)
    coop = nacc >= COOP_MIN_ACC
    split = (not coop) and nacc >= SPLIT_MIN_ACC
    if coop or split:
        src.append(emit_coop(name, coop_tables(la, lb, lc, ld)))
    src.append(f"struct {name} {{")
    src.append(f"  static constexpr bool COOP = {'true' if coop else 'false'};")
    src.append(f"  static constexpr bool SPLIT = {'true' if split else 'false'};")
    if coop or split:
        src.append(f"  using Coop = {name}Coop;")
    if split:
        sl, nch, _, perm = gen_vrr_split(la, lb, lc, ld)
        # a namespace-scope device table, like the other node tables
        src.insert(0, f"__device__ const unsigned short k{name}_perm[] = {{" + ", ".join(str(x) for x in perm) + "};")
        src.append(f"  static constexpr int NCHUNK = {nch};")
        src.append(f"  __device__ static const unsigned short* split_perm() {{ return k{name}_perm; }}")
        src.append("  template <typename R>")
        src.append("  __device__ __forceinline__ static void vrr_split(const R* __restrict__ G, const VrrGeo<R>& g,")
        src.append("                                                 R* __restrict__ acc, R* __restrict__ comp,")
        src.append("                                                 R* __restrict__ red) {")
        src.append("    const R PAx = g.PA[0], PAy = g.PA[1], PAz = g.PA[2];")
        src.append("    const R QCx = g.QC[0], QCy = g.QC[1], QCz = g.QC[2];")
        src.append("    const R WPx = g.WP[0], WPy = g.WP[1], WPz = g.WP[2];")
        src.append("    const R WQx = g.WQ[0], WQy = g.WQ[1], WQz = g.WQ[2];")
        src.append("    const R oo2p = g.oo2p, oo2q = g.oo2q, oo2pq = g.oo2pq, rop = g.rop, roq = g.roq;")
        src.append("    (void)PAx; (void)PAy; (void)PAz; (void)QCx; (void)QCy; (void)QCz;")
        src.append("    (void)WPx; (void)WPy; (void)WPz; (void)WQx; (void)WQy; (void)WQz;")
        src.append("    (void)oo2p; (void)oo2q; (void)oo2pq; (void)rop; (void)roq;")
        src.extend(sl)
        src.append("  }")
    src.append(f"  static constexpr int la = {la}, lb = {lb}, lc = {lc}, ld = {ld};")
    src.append(f"  static constexpr int bra_class = {ib}, ket_class = {ik};")
    src.append(f"  static constexpr int L = {la + lb + lc + ld};")
    src.append(f"  static constexpr int NA = {NA}, NB = {NB}, NC = {NC}, ND = {ND};")
    src.append(f"  static constexpr int NE = {len(v.E)}, NF = {len(v.F)}, NACC = {len(v.E) * len(v.F)};")
    src.append(f"  static constexpr int NOUT = {NA * NB * NC * ND};")
    src.append(f"  static constexpr int VRR_FLOPS = {v.flops}, HRR_FLOPS = {h.flops};")
    src.append(f"  static constexpr int PT_MIN_BLOCKS = {PT_MIN_BLOCKS.get((la, lb, lc, ld), 1)};")
    src.append(f"  static constexpr bool PT_PREFETCH = {'true' if (la, lb, lc, ld) in PT_PREFETCH else 'false'};")
    src.append(f"  static constexpr bool SPLIT_SMEM_ACC = {'true' if (la, lb, lc, ld) in SPLIT_SMEM_ACC else 'false'};")
    src.append(f"  static constexpr int SPLIT_WARPS = {SPLIT_WARPS.get((la, lb, lc, ld), 0)};")
    inl = "__forceinline__" if len(v.E) * len(v.F) <= INLINE_MAX_ACC else "__noinline__"
    src.append("  template <typename R>")
    src.append(f"  __device__ {inl} static void vrr(const R* __restrict__ G, const VrrGeo<R>& g, R* __restrict__ acc,")
    src.append("                                  R* __restrict__ comp) {")
    src.append("    const R PAx = g.PA[0], PAy = g.PA[1], PAz = g.PA[2];")
    src.append("    const R QCx = g.QC[0], QCy = g.QC[1], QCz = g.QC[2];")
    src.append("    const R WPx = g.WP[0], WPy = g.WP[1], WPz = g.WP[2];")
    src.append("    const R WQx = g.WQ[0], WQy = g.WQ[1], WQz = g.WQ[2];")
    src.append("    const R oo2p = g.oo2p, oo2q = g.oo2q, oo2pq = g.oo2pq, rop = g.rop, roq = g.roq;")
    src.append("    (void)PAx; (void)PAy; (void)PAz; (void)QCx; (void)QCy; (void)QCz;")
    src.append("    (void)WPx; (void)WPy; (void)WPz; (void)WQx; (void)WQy; (void)WQz;")
    src.append("    (void)oo2p; (void)oo2q; (void)oo2pq; (void)rop; (void)roq;")
    src.extend(vl)
    src.append("  }")
    src.append("  template <typename R>")
    src.append(f"  __device__ {inl} static void hrr(const R* __restrict__ acc, const R ABx, const R ABy, const R ABz,")
    src.append("                                             const R CDx, const R CDy, const R CDz, R* __restrict__ out) {")
    src.append("    (void)ABx; (void)ABy; (void)ABz; (void)CDx; (void)CDy; (void)CDz;")
    src.extend(hl)
    src.append("  }")
    src.append("};")
    info = dict(name=name, ib=ib, ik=ik, la=la, lb=lb, lc=lc, ld=ld, L=la + lb + lc + ld,
                nout=NA * NB * NC * ND, nacc=len(v.E) * len(v.F), vrr_flops=v.flops, hrr_flops=h.flops,
                kind=2 if coop else (1 if split else 0))
    return "\n".join(src), info


HEADER = """// GENERATED by gen_eri.py -- do not edit.  Per-class Obara-Saika/HGP ERI code.
#pragma once
#include "eri_common.cuh"
namespace hfx {
"""


def generate(outdir):
    os.makedirs(outdir, exist_ok=True)
    classes = quartet_classes()
    infos = []
    for (ib, ik, la, lb, lc, ld) in classes:
        src, info = gen_class(ib, ik, la, lb, lc, ld)
        infos.append(info)
        path = os.path.join(outdir, f"cls_{la}{lb}{lc}{ld}.cuh")
        _write_if_changed(path, HEADER + "\n" + src + "\n}  // namespace hfx\n")
    # class table (host + device readable)
    tab = ["// GENERATED by gen_eri.py -- do not edit.", "#pragma once",
           f"#define HFX_NCLASS {len(classes)}",
           "static const int hfx_class_table[HFX_NCLASS][12] = {",
           "  // bra_class, ket_class, la, lb, lc, ld, L, nout, vrr_flops, hrr_flops, n_acc,",
           "  // kernel kind (0 per-thread k_build_K, 1 split k_build_K_split, 2 cooperative k_build_K_coop)"]
    for c in infos:
        tab.append(f"  {{{c['ib']}, {c['ik']}, {c['la']}, {c['lb']}, {c['lc']}, {c['ld']}, {c['L']}, "
                   f"{c['nout']}, {c['vrr_flops']}, {c['hrr_flops']}, {c['nacc']}, {c['kind']}}},")
    tab.append("};")
    _write_if_changed(os.path.join(outdir, "class_table.h"), "\n".join(tab) + "\n")
    # launcher declarations and dispatch table, in class order
    dis = ["// GENERATED by gen_eri.py -- do not edit.", "#pragma once", "#include <cuda_runtime.h>",
           "#include \"class_table.h\"",
           "namespace hfx {", "struct BuildArgs;", "struct SchwarzArgs;", "struct EvalArgs;"]
    for c in infos:
        n = c["name"]
        dis.append(f"void launch_K_{n}(const BuildArgs&, int, int, cudaStream_t);")
        dis.append(f"int occupancy_K_{n}(int);")
        dis.append(f"void launch_schwarz_{n}(const SchwarzArgs&, cudaStream_t);")
        dis.append(f"void launch_eval_{n}(const EvalArgs&, int, cudaStream_t);")
    dis.append("struct ClassOps {")
    dis.append("  void (*launch_K)(const BuildArgs&, int, int, cudaStream_t);")
    dis.append("  int (*occupancy_K)(int);")
    dis.append("  void (*launch_schwarz)(const SchwarzArgs&, cudaStream_t);")
    dis.append("  void (*launch_eval)(const EvalArgs&, int, cudaStream_t);")
    dis.append("};")
    dis.append("static const ClassOps kClassOps[HFX_NCLASS] = {")
    for c in infos:
        n = c["name"]
        dis.append(f"  {{launch_K_{n}, occupancy_K_{n}, launch_schwarz_{n}, launch_eval_{n}}},")
    dis.append("};")
    dis.append("}  // namespace hfx")
    _write_if_changed(os.path.join(outdir, "class_dispatch.h"), "\n".join(dis) + "\n")
    # one translation unit per class
    for c in infos:
        n = f"{c['la']}{c['lb']}{c['lc']}{c['ld']}"
        tu = (f"// GENERATED by gen_eri.py -- do not edit.\n#include \"cls_{n}.cuh\"\n"
              f"#include \"eri_kernels.cuh\"\nHFX_INSTANTIATE_CLASS(Cls{n})\n")
        _write_if_changed(os.path.join(outdir, f"tu_{n}.cu"), tu)
    return infos


def _write_if_changed(path, text):
    if os.path.exists(path):
        with open(path) as fh:
            if fh.read() == text:
                return
    with open(path, "w") as fh:
        fh.write(text)




# ---------------------------------------------------------------- cooperative
# Large classes run the recursions cooperatively: one warp per contracted
# quartet, intermediates in shared memory, the DAG evaluated level by level
# from node tables.  A node is four 32-bit words:
#   x: dst | kind << 16 | axis << 18 | k1 << 20 | k2 << 24
#   y: s0 | s1 << 16,  z: s2 | s3 << 16,  w: s4
# kind 0 (bra VRR):  v = PA_i s0 + WP_i s1 + k1/(2p) (s2 - rho/p s3)
# kind 1 (ket VRR):  v = QC_i s0 + WQ_i s1 + k1/(2q) (s2 - rho/q s3) + k2/(2(p+q)) s4
# kind 2 (bra HRR):  v = s0 + AB_i s1;   kind 3 (ket HRR): v = s0 + CD_i s1
# VRR slots: 0 = constant zero, 1..L+1 = G_0..G_L, then nodes by level
# (level = |e| + |f|).  HRR slots: 0..NACC-1 = contracted [e0|f0], then nodes.
# Classes with at least this many accumulators use the cooperative
# (table-interpreter) kernel.  Measured on GB300 (100-atom HSE build): (dd|dd),
# 961 accumulators, runs 2.1x faster on the lockstep warp-split kernel, so by
# default no class does; HFX_COOP_MIN_ACC=900 brings it back for (dd|dd).
COOP_MIN_ACC = int(os.environ.get("HFX_COOP_MIN_ACC", "100000"))


def coop_tables(la, lb, lc, ld):
    v = VRR(la, lb, lc, ld)
    L = la + lb + lc + ld
    recs = {}  # (e, f, m) -> (kind, axis, k1, k2, srcs)

    def build(e, f, m):
        key = (e, f, m)
        if key in recs or (sum(e) == 0 and sum(f) == 0):
            return
        if sum(f) > 0:
            i = next(k for k in range(3) if f[k] > 0)
            f1 = _sub(f, i)
            srcs = [(e, f1, m), (e, f1, m + 1), None, None, None]
            k1 = f1[i]
            if k1 > 0:
                srcs[2], srcs[3] = (e, _sub(f1, i), m), (e, _sub(f1, i), m + 1)
            k2 = e[i]
            if k2 > 0:
                srcs[4] = (_sub(e, i), f1, m + 1)
            recs[key] = (1, i, k1, k2, srcs)
        else:
            i = next(k for k in range(3) if e[k] > 0)
            e1 = _sub(e, i)
            srcs = [(e1, f, m), (e1, f, m + 1), None, None, None]
            k1 = e1[i]
            if k1 > 0:
                srcs[2], srcs[3] = (_sub(e1, i), f, m), (_sub(e1, i), f, m + 1)
            recs[key] = (0, i, k1, 0, srcs)
        for s in recs[key][4]:
            if s is not None:
                build(*s)

    for e in v.E:
        for f in v.F:
            build(e, f, 0)
    slot = {}
    order = sorted(recs, key=lambda k: (sum(k[0]) + sum(k[1]), recs[k][0], k[2], k[0], k[1]))
    base = L + 2
    for n, k in enumerate(order):
        slot[k] = base + n

    def sidx(s):
        if s is None:
            return 0
        e, f, m = s
        if sum(e) == 0 and sum(f) == 0:
            return 1 + m
        return slot[s]

    nodes, lev_off = [], [0] * (L + 2)
    for k in order:
        kind, axis, k1, k2, srcs = recs[k]
        lev = sum(k[0]) + sum(k[1])
        lev_off[lev + 1] = len(nodes) + 1
        s = [sidx(x) for x in srcs]
        nodes.append((slot[k] | kind << 16 | axis << 18 | k1 << 20 | k2 << 24, s[0] | s[1] << 16,
                      s[2] | s[3] << 16, s[4]))
    # level offsets: lev_off[l] = first node of level l (levels 1..L)
    offs = [0] * (L + 2)
    cnt = [0] * (L + 2)
    for k in order:
        cnt[sum(k[0]) + sum(k[1])] += 1
    acc = 0
    for l in range(L + 2):
        offs[l] = acc
        acc += cnt[l]
    # first ket node of every level (bra nodes come first within a level)
    split = list(offs)
    for n, k in enumerate(order):
        lev = sum(k[0]) + sum(k[1])
        if recs[k][0] == 0:
            split[lev] = n + 1
    for l in range(L + 2):
        split[l] = max(split[l], offs[l])
    nf = len(v.F)
    targets = [sidx((e, f, 0)) for e in v.E for f in v.F]
    vrr_slots = base + len(order)
    vrr_flops_n = v.flops if False else None
    # horizontal recursion, bra then ket, as a DAG of kind-2/3 nodes
    E, F = v.E, v.F
    eidx = {e: i for i, e in enumerate(E)}
    fidx = {f: i for i, f in enumerate(F)}
    A_, B_, C_, D_ = comps(la), comps(lb), comps(lc), comps(ld)
    hnodes, hslot = [], {}
    nacc = len(E) * nf
    nxt = [nacc]
    hlev = {}

    def bslot(a, b, jf):
        if sum(b) == 0:
            return eidx[a] * nf + jf
        key = ("b", a, b, jf)
        if key in hslot:
            return hslot[key]
        i = next(k for k in range(3) if b[k] > 0)
        b1 = _sub(b, i)
        x, y = bslot(_add(a, i), b1, jf), bslot(a, b1, jf)
        hslot[key] = nxt[0]
        nxt[0] += 1
        hnodes.append(((hslot[key] | 2 << 16 | i << 18), x | y << 16, 0, 0, sum(b)))
        return hslot[key]

    def kslot(ia, ib, c, d):
        if sum(d) == 0:
            return bslot(A_[ia], B_[ib], fidx[c])
        key = ("k", ia, ib, c, d)
        if key in hslot:
            return hslot[key]
        i = next(k for k in range(3) if d[k] > 0)
        d1 = _sub(d, i)
        x, y = kslot(ia, ib, _add(c, i), d1), kslot(ia, ib, c, d1)
        hslot[key] = nxt[0]
        nxt[0] += 1
        hnodes.append(((hslot[key] | 3 << 16 | i << 18), x | y << 16, 0, 0, lb + sum(d)))
        return hslot[key]

    outs = []
    for ia in range(len(A_)):
        for ib in range(len(B_)):
            for c in C_:
                for d in D_:
                    outs.append(kslot(ia, ib, c, d))
    # HRR levels: bra nodes by |b| (1..lb), then ket nodes by lb + |d|
    nl = lb + ld
    hnodes, outs, hrr_slots = _reuse_hrr_slots(hnodes, outs, nacc, nl)
    hcnt = [0] * (nl + 2)
    for hn in hnodes:
        hcnt[hn[4]] += 1
    hnodes_sorted = sorted(hnodes, key=lambda hn: hn[4])
    hoffs, acc = [0] * (nl + 2), 0
    for l in range(nl + 2):
        hoffs[l] = acc
        acc += hcnt[l]
    return dict(nodes=nodes, lev_off=offs, lev_split=split, targets=targets, vrr_slots=vrr_slots,
                hnodes=[hn[:4] for hn in hnodes_sorted], hlev_off=hoffs, n_hlev=nl,
                hrr_slots=hrr_slots, outs=outs, nacc=nacc)


def _reuse_hrr_slots(hnodes, outs, nacc, nl):
    """Workspace slots of the horizontal recursion, reused once their value is
    dead.  The kernels run the nodes of one level in parallel (lanes) with a
    warp barrier between levels, so a slot read last at level l is free again
    for the nodes of level l + 1 on, and no level writes a slot it reads.  The
    contracted [e0|f0] stay in slots 0..nacc-1 (the epilogue writes them
    there); outputs stay live to the end.  Returns the renumbered nodes and
    outputs and the number of slots."""
    import heapq
    last = {}
    for xw, yw, _, _, lev in hnodes:
        for src in (yw & 0xFFFF, yw >> 16):
            last[src] = max(last.get(src, 0), lev)
    for o in outs:
        last[o] = nl + 1
    defined = {xw & 0xFFFF: lev for xw, _, _, _, lev in hnodes}
    # provisional slot -> the level before which it is released
    release = {}
    for sl in list(range(nacc)) + list(defined):
        release.setdefault(last.get(sl, defined.get(sl, 0)) + 1, []).append(sl)
    new = {sl: sl for sl in range(nacc)}
    free, top = [], nacc
    by_lev = {}
    for hn in hnodes:
        by_lev.setdefault(hn[4], []).append(hn)
    for lev in range(1, nl + 1):
        for l0 in range(lev + 1):
            for sl in release.pop(l0, []):
                heapq.heappush(free, new[sl])
        for hn in by_lev.get(lev, []):
            if free:
                d = heapq.heappop(free)
            else:
                d, top = top, top + 1
            new[hn[0] & 0xFFFF] = d
    out_nodes = []
    for xw, yw, zw, ww, lev in hnodes:
        a, b = new[yw & 0xFFFF], new[yw >> 16]
        out_nodes.append(((xw & ~0xFFFF) | new[xw & 0xFFFF], a | b << 16, zw, ww, lev))
    # no level writes a slot that the same level reads or writes twice
    for lev in range(1, nl + 1):
        ws = [hn[0] & 0xFFFF for hn in out_nodes if hn[4] == lev]
        rs = {s for hn in out_nodes if hn[4] == lev for s in (hn[1] & 0xFFFF, hn[1] >> 16)}
        assert len(ws) == len(set(ws)) and not (set(ws) & rs), lev
    return out_nodes, [new[o] for o in outs], top


def emit_coop(name, t):
    def arr(tp, nm, vals):
        body = ", ".join(str(x) for x in vals) if vals else "0"
        return f"__device__ const {tp} {nm}[] = {{{body}}};"

    def arr4(nm, vals):
        body = ", ".join(f"{{{a}u, {b}u, {c}u, {d}u}}" for (a, b, c, d) in vals) if vals else "{0u, 0u, 0u, 0u}"
        return f"__device__ const uint4 {nm}[] = {{{body}}};"

    lines = [arr4(f"k{name}_vrr", t["nodes"]), arr("int", f"k{name}_vlev", t["lev_off"]),
             arr("int", f"k{name}_vsplit", t["lev_split"]),
             arr("unsigned short", f"k{name}_tgt", t["targets"]), arr4(f"k{name}_hrr", t["hnodes"]),
             arr("int", f"k{name}_hlev", t["hlev_off"]), arr("unsigned short", f"k{name}_out", t["outs"])]
    lines.append(f"struct {name}Coop {{")
    lines.append(f"  static constexpr int VRR_SLOTS = {t['vrr_slots']}, HRR_SLOTS = {t['hrr_slots']};")
    lines.append(f"  static constexpr int N_VLEV = {len(t['lev_off']) - 1}, N_HLEV = {t['n_hlev']};")
    lines.append(f"  __device__ static const uint4* vrr() {{ return k{name}_vrr; }}")
    lines.append(f"  __device__ static const int* vlev() {{ return k{name}_vlev; }}")
    lines.append(f"  __device__ static const int* vsplit() {{ return k{name}_vsplit; }}")
    lines.append(f"  __device__ static const unsigned short* tgt() {{ return k{name}_tgt; }}")
    lines.append(f"  __device__ static const uint4* hrr() {{ return k{name}_hrr; }}")
    lines.append(f"  __device__ static const int* hlev() {{ return k{name}_hlev; }}")
    lines.append(f"  __device__ static const unsigned short* out() {{ return k{name}_out; }}")
    lines.append("};")
    return "\n".join(lines)



# ---------------------------------------------------------------- split
# Medium-large classes run one warp per shell quartet with the lanes on
# different primitive quartets: each lane evaluates the straight-line vertical
# recursion of its own primitive quartet, and every 32 finished targets are
# summed over the warp by a butterfly reduce-scatter, after which lane j holds
# target (32 k + j).  The targets are emitted e-major (accumulator order) in a
# depth-first order, which keeps the live set of the recursion small.
SPLIT_MIN_ACC = 90

# Target order of the warp-split vertical recursion: "grouped"
# (_grouped_target_order, the default) or "greedy" (_greedy_target_order).
# The grouped order holds fewer values live at once; ptxas reports it cuts the
# spill stores of the (dd|dd) kernels from 34 322 to 13 454 bytes (FP64) and
# from 10 858 to 1 394 bytes (FP32).  HFX_VRR_ORDER selects it at build time.
VRR_ORDER = os.environ.get("HFX_VRR_ORDER", "grouped")


def _greedy_target_order(v, targets):
    """Targets in an order that keeps the recursion's live set small: at each
    step the target whose evaluation needs the fewest not-yet-computed nodes."""
    deps = {}

    def srcs(e, f, m):
        out = []
        if sum(f) > 0:
            i = next(k for k in range(3) if f[k] > 0)
            f1 = _sub(f, i)
            out += [(e, f1, m), (e, f1, m + 1)]
            if f1[i] > 0:
                out += [(e, _sub(f1, i), m), (e, _sub(f1, i), m + 1)]
            if e[i] > 0:
                out += [(_sub(e, i), f1, m + 1)]
        elif sum(e) > 0:
            i = next(k for k in range(3) if e[k] > 0)
            e1 = _sub(e, i)
            out += [(e1, f, m), (e1, f, m + 1)]
            if e1[i] > 0:
                out += [(_sub(e1, i), f, m), (_sub(e1, i), f, m + 1)]
        return [x for x in out if sum(x[0]) + sum(x[1]) > 0]

    def collect(k):
        if k in deps:
            return
        deps[k] = srcs(*k)
        for x in deps[k]:
            collect(x)

    for (e, f) in targets:
        collect((e, f, 0))
    done, order, left = set(), [], list(targets)

    def closure(k, acc):
        if k in done or k in acc:
            return
        for x in deps[k]:
            closure(x, acc)
        acc.add(k)

    while left:
        best = None
        for t in left:
            acc = set()
            closure((t[0], t[1], 0), acc)
            if best is None or len(acc) < best[0]:
                best = (len(acc), t, acc)
        done |= best[2]
        order.append(best[1])
        left.remove(best[1])
    return order


def _node_sources(e, f, m):
    """The recursion nodes (e', f', m') that node (e, f, m) reads (the
    Obara-Saika steps of VRR.node; the G_m leaves left out)."""
    out = []
    if sum(f) > 0:
        i = next(k for k in range(3) if f[k] > 0)
        f1 = _sub(f, i)
        out += [(e, f1, m), (e, f1, m + 1)]
        if f1[i] > 0:
            out += [(e, _sub(f1, i), m), (e, _sub(f1, i), m + 1)]
        if e[i] > 0:
            out += [(_sub(e, i), f1, m + 1)]
    elif sum(e) > 0:
        i = next(k for k in range(3) if e[k] > 0)
        e1 = _sub(e, i)
        out += [(e1, f, m), (e1, f, m + 1)]
        if e1[i] > 0:
            out += [(_sub(e1, i), f, m), (_sub(e1, i), f, m + 1)]
    return [x for x in out if sum(x[0]) + sum(x[1]) > 0]


def _grouped_target_order(v, targets, bonus_group=4.0, bonus_target=1.0):
    """Targets grouped by their bra index e.  The groups, and then the targets
    inside each group, are picked one at a time: the one whose evaluation needs
    the fewest not-yet-computed nodes, less a bonus for every computed node it
    lets go (all of that node's users are then computed).  Smaller peak live
    set than _greedy_target_order for the d-shell classes."""
    deps = {}

    def collect(k):
        if k in deps:
            return
        deps[k] = _node_sources(*k)
        for x in deps[k]:
            collect(x)

    for (e, f) in targets:
        collect((e, f, 0))
    users = {}
    for k, ds in deps.items():
        for x in set(ds):
            users.setdefault(x, set()).add(k)

    def cone(k, acc):
        if k in acc:
            return
        acc.add(k)
        for x in deps[k]:
            cone(x, acc)

    tcone = {}
    for t in targets:
        a = set()
        cone((t[0], t[1], 0), a)
        tcone[t] = a

    def pick(items, cone_of, done, bonus):
        order, left = [], list(items)
        while left:
            best = None
            for it in left:
                acc = cone_of(it) - done
                da = done | acc
                freed = sum(1 for x in acc for y in deps[x] if y in done and users[y] <= da)
                score = len(acc) - bonus * freed
                if best is None or score < best[0]:
                    best = (score, it, acc)
            done |= best[2]
            order.append(best[1])
            left.remove(best[1])
        return order

    es = sorted({t[0] for t in targets}, key=lambda e: (sum(e), e))
    fs = [t[1] for t in targets if t[0] == targets[0][0]]
    group = {e: set().union(*(tcone[(e, f)] for f in fs)) for e in es}
    e_order = pick(es, lambda e: group[e], set(), bonus_group)
    done, out = set(), []
    for e in e_order:
        out += pick([(e, f) for f in fs], lambda t: tcone[t], done, bonus_target)
    return out


def gen_vrr_split(la, lb, lc, ld):
    v = VRR(la, lb, lc, ld)
    nf = len(v.F)
    eidx = {e: i for i, e in enumerate(v.E)}
    fidx = {f: i for i, f in enumerate(v.F)}
    order = _grouped_target_order if VRR_ORDER == "grouped" else _greedy_target_order
    targets = order(v, [(e, f) for e in v.E for f in v.F])
    perm = [eidx[e] * nf + fidx[f] for (e, f) in targets]
    lines = []
    emitted_before = 0
    nch = (len(targets) + 31) // 32
    for k in range(nch):
        chunk = targets[32 * k: 32 * (k + 1)]
        names = [v.node(e, f, 0) for (e, f) in chunk]
        new = v.lines[emitted_before:]
        emitted_before = len(v.lines)
        lines.extend(new)
        vals = names + ["R(0)"] * (32 - len(names))
        lines.append("    {")
        lines.append("      R c_[32] = {" + ", ".join(vals) + "};")
        lines.append(f"      kacc<R>(acc[{k}], comp[{k}], chunk_reduce32<R>(c_, red));")
        lines.append("    }")
    v.flops += len(targets)
    return lines, nch, v.flops, perm


if __name__ == "__main__":
    out = sys.argv[1] if len(sys.argv) > 1 else os.path.join(os.path.dirname(__file__), "generated")
    for c in generate(out):
        print(c)
