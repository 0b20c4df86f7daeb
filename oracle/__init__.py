"""CPU oracle for basic and one-line full ORBGRAND (arXiv 2202.13951).

TEST INFRASTRUCTURE ONLY: the tests, ``__graft_entry__.smoke()`` and the
benchmark's CPU-baseline leg may use it; the product path never does.
It shares no code with the CUDA library.

Functions and the passages they follow:
  decode / decode_batch  Algorithm 1 with the basic ORBGRAND generator
                         (Sec. III-A/B, Eq. lw, Eq. fractionation,
                         Eq. intpart2, Eq. vu, Algorithm 2)
  enumerate_patterns     the query order itself (Sec. III-B, Algorithm 2)
  count_by_weight        patterns per (W, w) met by that order
  landslide              Algorithm 2 with Build-mountain (Sec. III-C)
  sort_reliability       the permutation pi (Sec. III-A)
  decode_1line / decode_batch_1line / enumerate_patterns_1line
                         one-line full ORBGRAND (Sec. III-D, Eq. relest_seg
                         with m = 1, Eq. wu_i): the order of increasing
                         reliability weight J0 w_H + beta w_L
  decode_batch_mline / enumerate_patterns_mline
                         m-segment full ORBGRAND (Sec. III-D: Eq.
                         relest_seg, Algorithm 3 splits checked by
                         Algorithm 4 / Eq. wi_cond, Landslide per segment,
                         the Cartesian product of Eq. cartP)
  fit                    piece-wise linear fitting and quantisation of a
                         block's ordered reliabilities (Sec. III-E, Eq. Q,
                         Eq. quant)
  decode_batch_fit       full ORBGRAND per block: fit, then the m-segment
                         order

Parity pins: tests/test_oracle_pins.py (brute force on tiny codes, the
first queries of Sec. III-B, the Fig. 3 / Fig. 5 examples, closed-form
partition counts, decoder invariants), tests/test_oracle_1line.py (the
one-line order against brute force and its generating function; J0 = 0,
beta = 1 is basic ORBGRAND) and tests/test_oracle_mutations.py (planted
mistakes must fail a pin).
"""
from .oracle import (Oracle, OracleError, build_oracle, compile_oracle,
                     count_by_weight, decode, decode_1line, decode_batch,
                     decode_batch_1line, decode_batch_mline, default,
                     enumerate_patterns, enumerate_patterns_1line,
                     enumerate_patterns_mline, fit, decode_batch_fit, landslide,
                     sort_reliability, ORACLE_LIB, ORACLE_SRC)

__all__ = ["Oracle", "OracleError", "build_oracle", "compile_oracle",
           "count_by_weight", "decode", "decode_1line", "decode_batch",
           "decode_batch_1line", "decode_batch_mline", "default",
           "enumerate_patterns", "enumerate_patterns_1line",
           "enumerate_patterns_mline", "fit", "decode_batch_fit", "landslide",
           "sort_reliability", "ORACLE_LIB", "ORACLE_SRC"]
