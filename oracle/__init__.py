"""Plain, slow CPU oracle of RNS-CKKS and of the paper's sharded convolution and pooling.

TEST INFRASTRUCTURE ONLY.  Only tests/, ``__graft_entry__.smoke()`` and bench.py's
CPU-baseline leg (including ``bench.py --impl reference``) may import or run anything here.
It shares no code, table or constant generator with the CUDA path in
``paper_2306_09189_gb300``; neither imports the other.

Modules: params (primes), encode (canonical embedding), ckks (scheme), layers (Sec. 4 layer
programs and their cleartext slot simulator), bootstrap (ModRaise, CoeffToSlot, EvalMod,
SlotToCoeff), ckks_ref.c (the u128 `%` ring arithmetic).

Pins (tests/test_oracle_*.py): schoolbook negacyclic products and direct evaluation for the
NTT; exact big-integer CRT identities for fast base conversion, ModDown and rescale; the naive
DFT for the encoder; np.roll for rotations; elementwise products for relinearisation;
torch conv2d/avg_pool2d for the layer plans; the paper's Chebyshev-node error table
(Appendix, polynomial approximation) for the interpolation routine; for bootstrapping the dense
encoding matrix, the exact ModRaise identity, conjugated and rotated decryptions, and the
decrypted message after a whole bootstrap.
"""
