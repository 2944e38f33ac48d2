"""FASTA input for queries and databases.

``read`` parses FASTA text (a path, a file object or the text itself) into
record names and one concatenated, encoded SeqSet, ready for
``swgb.Database`` and ``Plan.search``.  Residues are encoded by the library's
own ``sw_encode`` (BLOSUM62 order, a-z folded, U/O/J and unknown letters to
X); white space inside a sequence is skipped.
"""
from __future__ import annotations

import io
import os

import numpy as np

from . import swgb
from .synth import SeqSet


def _lines(src):
    if hasattr(src, "read"):
        return io.StringIO(src.read())
    if isinstance(src, (str, os.PathLike)) and os.path.exists(src):
        with open(src, encoding="latin-1") as fh:
            return io.StringIO(fh.read())
    return io.StringIO(str(src))


def read(src) -> tuple[list[str], SeqSet]:
    """(names, sequences) of every record, in file order.  A name is the
    header line after '>' up to the first white space.  Text before the first
    header is an error; a record may be empty."""
    names, seqs, cur = [], [], None
    for ln in _lines(src):
        ln = ln.rstrip("\r\n")
        if ln.startswith(">"):
            if cur is not None:
                seqs.append("".join(cur))
            head = ln[1:].strip()
            names.append(head.split()[0] if head else "")
            cur = []
        elif ln.strip():
            if cur is None:
                raise ValueError("FASTA text before the first '>' header")
            cur.append("".join(ln.split()))
    if cur is not None:
        seqs.append("".join(cur))
    lens = np.array([len(s) for s in seqs], dtype=np.int32)
    res = swgb.encode("".join(seqs)) if lens.sum() else np.zeros(0, np.uint8)
    return names, SeqSet(res, lens)
