"""FASTA input: records, names, multi-line sequences and encoding through the
library's sw_encode (checked against the oracle's encoder)."""
import io

import numpy as np
import pytest

import oracle
from paper_2309_09609_gb300 import build as nvbuild
from paper_2309_09609_gb300 import fasta


@pytest.fixture(scope="module", autouse=True)
def built():
    nvbuild.build()


TEXT = """>first made-up record
MKTAYIAK
QRQISFVK
>second
acdefghik  lmnp

>empty
>last description with spaces
WUXBZ*
"""


def test_records_names_and_codes(tmp_path):
    names, ss = fasta.read(TEXT)
    assert names == ["first", "second", "empty", "last"]
    assert ss.lens.tolist() == [16, 13, 0, 6]
    want = ["MKTAYIAKQRQISFVK", "acdefghiklmnp", "", "WUXBZ*"]
    for i, w in enumerate(want):
        assert (ss.seq(i) == oracle.encode(w)).all(), i
    # the same from a path and from a file object
    p = tmp_path / "x.fasta"
    p.write_text(TEXT)
    for src in (str(p), p, io.StringIO(TEXT)):
        n2, s2 = fasta.read(src)
        assert n2 == names and (s2.res == ss.res).all() and (s2.lens == ss.lens).all()


def test_edge_cases():
    names, ss = fasta.read("")
    assert names == [] and len(ss) == 0 and ss.res.size == 0
    names, ss = fasta.read(">only\n")
    assert names == ["only"] and ss.lens.tolist() == [0]
    with pytest.raises(ValueError):
        fasta.read("MKT\n>late header\nAAA\n")
    names, ss = fasta.read(">\nAC\r\n>b\r\nD\r\n")       # empty name, CRLF line ends
    assert names == ["", "b"] and ss.lens.tolist() == [2, 1]
    assert ss.res.dtype == np.uint8 and ss.res.max() < 24
