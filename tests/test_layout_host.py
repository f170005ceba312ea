"""Host-side checks of the CUDA path's index and sizing functions, without a GPU.

tests/layout_values.cu prints the values the kernels compute with their host-callable layout functions (column
chunk counts and offsets, half-chunk work items, reversed-column offsets of theta, the witness index, workspace
strides, shared-memory sizes). This file checks them against sums and counts formed here from the definitions.
"""
import itertools
import json
import math
import os
import shutil
import subprocess

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
CSRC = os.path.join(ROOT, "paper_2502_12428_gb300", "csrc")
MAX_SMEM = 227 * 1024   # dynamic shared memory one CTA may opt into


def _nvcc():
    cand = os.path.join(os.environ.get("CUDA_HOME", "/usr/local/cuda"), "bin", "nvcc")
    return cand if os.path.exists(cand) else shutil.which("nvcc")


@pytest.fixture(scope="module")
def values(tmp_path_factory):
    nvcc = _nvcc()
    if not nvcc:
        pytest.skip("nvcc not found")
    exe = str(tmp_path_factory.mktemp("layout") / "layout_values")
    subprocess.run([nvcc, "-gencode", "arch=compute_103a,code=sm_103a", "-std=c++17", "-I", CSRC,
                    "-I", os.path.join(ROOT, "include"), os.path.join(ROOT, "tests", "layout_values.cu"), "-o", exe],
                   check=True, capture_output=True)
    out = subprocess.run([exe], check=True, capture_output=True, text=True).stdout
    return json.loads(out)


def test_columns_are_sized_for_s_plus_4(values):
    # column s holds the residues t = 0..s and at least four zero bytes after them, so its last word is padding
    for s, c in enumerate(values["chunks_of"]):
        assert c == (s + 4) // 16 + 1
        assert 16 * c - 4 >= s + 1


def test_column_offsets_are_running_sums(values):
    ch = values["chunks_of"]
    assert values["chunk_prefix"] == [sum(ch[:s]) for s in range(len(ch))]
    assert values["half_prefix"] == [sum(x // 8 + 1 for x in range(s)) for s in range(len(ch))]
    assert values["rcolw"] == [sum(x // 4 + 1 for x in range(s)) for s in range(len(values["rcolw"]))]


def descending_lex(deg):
    for e1 in range(deg, -1, -1):
        for e2 in range(deg - e1, -1, -1):
            for e3 in range(deg - e1 - e2, -1, -1):
                yield (e1, e2, e3, deg - e1 - e2 - e3)


@pytest.mark.parametrize("p", [3, 5, 7, 11, 13])
def test_prime_constants(values, p):
    v = values["primes"][str(p)]
    d, D = 4 * (p - 1), 4 * p * (p - 1)
    assert (v["d"], v["D"]) == (d, D)
    assert v["ld"] == math.comb(d + 3, 3) and v["lD"] == math.comb(D + 3, 3)
    # the witness monomial (x1 x2 x3 x4)^(p-1) of Fedder's test, in descending-lex order of degree d
    target = (p - 1,) * 4
    assert v["witness"] == next(i for i, m in enumerate(descending_lex(d)) if m == target)


@pytest.mark.parametrize("p", [3, 5, 7, 11, 13])
def test_workspace_and_shared_memory_fit(values, p):
    v = values["primes"][str(p)]
    D = v["D"]
    ch = values["chunks_of"]
    # a padded form of degree D: slice u holds the columns s = 0..u
    padded_words = sum(4 * sum(ch[: u + 1]) for u in range(D + 1))
    assert v["stride"] >= padded_words
    assert v["smem_sweep"] <= MAX_SMEM and v["smem_ring"] <= MAX_SMEM


def test_published_form_sizes(values):
    # C(4p-1, 3) and C(4p(p-1)+3, 3) as the configurations state them
    sizes = {p: (values["primes"][str(p)]["ld"], values["primes"][str(p)]["lD"]) for p in (3, 5, 7, 11)}
    assert sizes == {3: (165, 2925), 5: (969, 91881), 7: (2925, 818805), 11: (12341, 14391741)}
    assert sum(1 for _ in itertools.islice(descending_lex(4), 100)) == 35


def test_integer_index_decoders(values):
    # isqrt / icbrt around every square and cube, and the item, chunk and packed-index decoders over every index
    # up to the largest degree, against enumeration: integer arithmetic only, no mismatch
    m = values["decoder_mismatches"]
    assert m["packed_entries"] == math.comb(values["max_d"] + 3, 3)
    assert {k: v for k, v in m.items() if k != "packed_entries"} == {"isqrt": 0, "icbrt": 0, "half": 0, "chunk": 0,
                                                                      "packed": 0}


def test_chain_reduction_by_multiply_high(values):
    # the chain's outputs reduce mod p^2 by one multiply-high; it equals a % p^2 for every value a chain output
    # can take (35 products of a residue below p^2 and a coefficient below p)
    assert values["mod_mismatches"] == [0, 0, 0, 0, 0]
