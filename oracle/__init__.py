"""CPU oracle for the Cascading Haar Wavelet (CHW) Walsh-Hadamard transform.

TEST INFRASTRUCTURE ONLY.  Nothing in the product path (the CUDA library and its
Python binding) may import, call or link anything in this package.  Only the test
suite, the smoke check of ``__graft_entry__`` and the CPU-baseline leg of
``bench.py`` use it.  It shares no code, table or constant with the CUDA path:
every constant (1/sqrt2, 2^(-m/2), the bit reversal) is recomputed here from its
mathematical definition.

What it computes (paper: "The Cascading Haar Wavelet algorithm for computing the
Walsh-Hadamard Transform", arXiv 1609.06641):

* ``definitions``  -- the matrices of eq. (1) (dyadic Hadamard H_m) and eq. (2)
  (Haar Psi_m), the stage factors of Theorem 1, the Haar-Walsh block structure of
  eq. (4), and the closed form of H_m's entries derived from eq. (1).  FP64 / int64.
* ``transforms``   -- the transform itself in three independent ways: the dense
  matvec (O1), a textbook natural-order fast WHT followed by a bit-reversal
  reorder (O2), and the closed form one entry at a time (O3, also vectorised over
  sampled outputs for sparse inputs, for signals too long to transform on the
  host); plus the CHW
  cascade of Theorem 1 taken literally in stage order (O4, any dtype, with an
  operation counter for Lemma 1 / Theorem 2) and its transpose, the reversed
  cascade of inverse Haar transforms.
* ``wavelets``     -- the Haar transform Psi_m of eq. (2), its transpose, and the
  Haar-Walsh transform H_m Psi_m^T of eq. (4) (stages 1..m-1 of Theorem 1).
* ``orderings``    -- natural (Sylvester) and sequency (Walsh) orderings of the outputs.
* ``lowp``         -- the bf16/fp16 storage form: per-signal power-of-two
  exponents decided in fp32, the same precision the kernels decide them in.
* ``errors``       -- FP64 normwise relative error per signal.

Parity pinned for: every function here (see tests/test_oracle_pins.py and
tests/test_oracle_mutations.py).  Parity unpinned: none.
"""

from .definitions import (
    hadamard_dyadic,
    haar_matrix,
    cascade_stage_factor,
    cascade_product,
    haar_walsh_blockdiag,
    bitrev,
    hadamard_entry_closed_form,
)
from .transforms import (
    wht_dense,
    wht_fast_dyadic,
    wht_closed_form,
    wht_sparse_closed_form,
    haar_analysis,
    haar_synthesis,
    chw_cascade,
    chw_reverse_cascade,
    OpCounter,
    end_scale_f32,
    inv_sqrt2,
)
from .wavelets import haar_forward, haar_inverse, haar_levels, haar_walsh
from .orderings import hadamard_natural, order_permutation, sign_changes, walsh_sequency_matrix, wht_ordered
from .lowp import codes_to_f32, dequantise, lowp_forward_reference, round_to_bf16, round_to_f16
from .errors import rel_err_per_signal

__all__ = [
    "hadamard_dyadic",
    "haar_matrix",
    "cascade_stage_factor",
    "cascade_product",
    "haar_walsh_blockdiag",
    "bitrev",
    "hadamard_entry_closed_form",
    "wht_dense",
    "wht_fast_dyadic",
    "wht_closed_form",
    "wht_sparse_closed_form",
    "haar_analysis",
    "haar_synthesis",
    "chw_cascade",
    "chw_reverse_cascade",
    "OpCounter",
    "end_scale_f32",
    "inv_sqrt2",
    "hadamard_natural",
    "order_permutation",
    "sign_changes",
    "walsh_sequency_matrix",
    "wht_ordered",
    "haar_forward",
    "haar_inverse",
    "haar_levels",
    "haar_walsh",
    "lowp_forward_reference",
    "round_to_bf16",
    "round_to_f16",
    "dequantise",
    "codes_to_f32",
    "rel_err_per_signal",
]
