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
