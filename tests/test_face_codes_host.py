"""Host logic of the 3-D face codes (CPU only): which cells near domain faces
the coded form of the step takes, and their codes, on small geometries whose
answer follows from the boundary rules by hand.

The coded form applies the inlet (Eq. 31) and outlet (Eq. 32, constant
pressure) rules per population and face ghosts on the lines; the general
form keeps the cells where it would bounce a face-crossing population back
(a solid boundary column, found with the periodic axes wrapped), where the
Eq. 32 inner cell is solid, and those that reach the faces of two axes or a
wall face."""
import json
import os
import shutil
import subprocess

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
CSRC = os.path.join(ROOT, "paper_2304_05657_gb300", "csrc")


@pytest.fixture(scope="module")
def cases(tmp_path_factory):
    nvcc = shutil.which("nvcc") or "/usr/local/cuda/bin/nvcc"
    if not os.path.exists(nvcc):
        pytest.skip("nvcc not found")
    out = tmp_path_factory.mktemp("face_codes") / "face_codes_cases"
    cmd = [nvcc, "-gencode", "arch=compute_103a,code=sm_103a", "-O1", "-std=c++17", "--expt-relaxed-constexpr",
           "-I", CSRC, "-I", os.path.join(ROOT, "include"), os.path.join(ROOT, "tests", "host", "face_codes_cases.cu"),
           os.path.join(CSRC, "lbfd_step.cu"), "-o", str(out)]
    subprocess.run(cmd, check=True, capture_output=True)
    res = subprocess.run([str(out)], check=True, capture_output=True, text=True)
    return {d["case"]: d for d in (json.loads(line) for line in res.stdout.splitlines())}


def xyz(d, c):
    return c % d["nx"], (c // d["nx"]) % d["ny"], c // (d["nx"] * d["ny"])


def test_open_faces_all_coded(cases):
    d = cases["open"]
    assert d["rest"] == []
    assert len(d["coded"]) == 4 * 6 * 5  # x in {0, 1, 10, 11}
    for c, code in d["coded"]:
        x, _, _ = xyz(d, c)
        # x axis: ghost distance on the side of the face (low 3 bits: -,
        # high 3 bits: +), and the face flag of that side; nothing else
        expect = {0: (1 << 32) | (1 << 50), 1: (2 << 32) | (1 << 50),
                  10: (2 << 35) | (1 << 51), 11: (1 << 35) | (1 << 51)}[x]
        assert code == expect, (x, hex(code))


def test_solid_column_across_a_periodic_seam(cases):
    # solid (0, 5, 0): populations (+1, c_y, c_z) of the inlet cells (0, y, z)
    # cross the inlet face with the boundary column (0, y - c_y, z - c_z)
    # wrapped in y and z; it is the solid cell for y in {4, 5, 0} and
    # z in {4, 0, 1}
    d = cases["seam"]
    rest = sorted(xyz(d, c) for c in d["rest"])
    expect = sorted((0, y, z) for y in (4, 5, 0) for z in (4, 0, 1) if (y, z) != (5, 0))
    assert rest == expect
    coded = {xyz(d, c): code for c, code in d["coded"]}
    # (1, 5, 0) pulls population (+1, 0, 0) (index 2 + 3 + 9 = 14) from the
    # solid: bounce-back; its x line meets the solid at distance 1 (not a
    # face)
    code = coded[(1, 5, 0)]
    assert (code >> 14) & 1 == 1 and code & ((1 << 27) - 1) == 1 << 14
    assert (code >> 32) & 0x3F == 1 and (code >> 50) & 0x3F == 0
    # (0, 5, 2): the inlet face at distance 1 on its x line, the solid at
    # distance 2 on the low side of its z line
    code = coded[(0, 5, 2)]
    assert (code >> 32) & 0x3F == 1 and (code >> 50) & 3 == 1
    assert (code >> 44) & 0x3F == 2 and (code >> 54) & 3 == 0


def test_solid_inner_cell_of_the_convective_outlet(cases):
    # Eq. 32 takes the inner cell (x - 1) of an outlet cell; solid there, the
    # general form keeps the cell; the constant-pressure outlet has no inner
    # cell
    d = cases["inner_eq32"]
    assert sorted(xyz(d, c) for c in d["rest"]) == [(11, 2, 2)]
    assert cases["inner_pressure"]["rest"] == []


def test_wall_faces_stay_with_the_general_form(cases):
    d = cases["walls_y"]
    coded = sorted(xyz(d, c) for c, _ in d["coded"])
    assert coded == sorted((x, y, z) for x in (0, 1, 10, 11) for y in range(2, 6) for z in range(5))
    assert len(d["rest"]) == 12 * 4 * 5  # every cell within two of a y wall


def test_wall_codes_around_one_solid_cell(cases):
    """Every cell within reach of a single solid cell at (4, 4, 4) of a
    periodic 9^3 domain: bounce-back bits for the populations pulled from it
    (the cell at x - c_i is the solid) and, on each axis line through the
    solid, the distance of the ghost on the solid's side."""
    d = cases["one_solid"]
    codes = {xyz(d, c): code for c, code in d["coded"]}
    # the listed cells: the 26 neighbours and the 6 axis cells at distance 2
    assert len(codes) == 26 + 6
    s = (4, 4, 4)
    for (x, y, z), code in codes.items():
        dx, dy, dz = x - s[0], y - s[1], z - s[2]
        bits = code & ((1 << 27) - 1)
        if max(abs(dx), abs(dy), abs(dz)) == 1:
            # population c = (dx, dy, dz) comes from the solid
            i = (dx + 1) + 3 * (dy + 1) + 9 * (dz + 1)
            assert bits == 1 << i, ((x, y, z), hex(bits))
        else:
            assert bits == 0
        for a, dist in enumerate((dx, dy, dz)):
            line = (code >> (32 + 6 * a)) & 0x3F
            others = [v for b, v in enumerate((dx, dy, dz)) if b != a]
            if others == [0, 0] and dist != 0:
                side_bits = abs(dist) << 3 if dist < 0 else abs(dist)  # dist < 0: the solid is on the + side
                assert line == side_bits, ((x, y, z), a, line)
            else:
                assert line == 0, ((x, y, z), a, line)
        assert (code >> 50) == 0
