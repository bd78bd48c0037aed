"""Source-level checks of the CUDA library (no GPU): the batched stage kernel
builds its stage parameters field by field in device code, without zeroing
them, so every field the stage tile reads must be assigned there.  A field
added to StageParams and read by the tile but forgotten in the batch body
would be an uninitialised value on the device (a pointer written through)."""
import os
import re

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
CSRC = os.path.join(ROOT, "paper_1711_01175_gb300", "csrc")


def _read(name):
    with open(os.path.join(CSRC, name)) as f:
        return f.read()


def test_batch_body_sets_every_stage_parameter_the_tile_reads():
    stage = _read("dgw_stage.cuh")
    head = _read("dgw_internal.cuh")
    start = head.index("struct StageParams {")
    fields = set()
    for line in head[start:head.index("};", start)].splitlines()[1:]:
        fields.update(re.findall(r"(\w+)(?:\[[^\]]*\])?\s*[,;]", line.split("//")[0]))
    body = stage[stage.index("void stage_batch_body"):stage.index("stage_tile<N, Real, kModeLsrk>(ps,")]
    assigned = set(re.findall(r"\bps\.(\w+)\s*=", body))
    tile = stage[stage.index("void stage_tile("):stage.index("void stage_kernel_body(")]
    read = set(re.findall(r"\bp\.(\w+)", tile)) & fields
    assert read, "no stage parameters found"
    assert not (read - assigned), sorted(read - assigned)


def test_l2_prefetch_is_off_exactly_where_the_l1_prefetch_runs():
    """The FP32 CUDA-core stage either prefetches the neighbour traces into L1
    (l1_prefetch) or prefetches later tiles into L2 (stage_pf_tenths): an L2
    prefetch ahead evicts the traces the L1 form is about to gather, so the two
    are chosen per degree as a pair.  The mixed table must be zero at exactly
    the degrees the L1 form is compiled for."""
    stage = _read("dgw_stage.cuh")
    head = _read("dgw_internal.cuh")
    m = re.search(r"constexpr bool l1_prefetch\(\) \{\s*return std::is_same<Real, float>::value && "
                  r"VOL == kVolCuda && \(([^;]*)\);", stage)
    assert m, "l1_prefetch condition not found"
    cond = m.group(1).replace("||", " or ").replace("&&", " and ")
    l1 = {N for N in range(1, 8) if eval(cond, {"__builtins__": {}, "N": N})}
    t = re.search(r"static const int kMixed\[8\] = \{([^}]*)\};", head)
    assert t, "mixed prefetch table not found"
    tenths = [int(v) for v in t.group(1).split(",")]
    assert len(tenths) == 8
    assert {N for N in range(1, 8) if tenths[N] == 0} == l1
    assert l1 == {3, 5, 6, 7}
