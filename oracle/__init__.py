"""FP64 CPU oracle for Electric Vertex Splitting (EVS) and the Virtual Transmission Method (VTM).

TEST INFRASTRUCTURE ONLY.  This package is the plain, slow, obviously-correct reference that the
CUDA path is checked against.  Only ``tests/``, ``__graft_entry__.smoke()`` and the CPU-baseline
and reference legs of ``bench.py`` may import it.  The product path (``paper_0807_1949_gb300``) never imports,
calls or links it, and it shares no code with the product beyond the seeded input generators
in ``paper_0807_1949_gb300/inputs.py`` (which hold none of the method's arithmetic).

Modules, each following the paper in its own order and notation:

* ``evs``      — §4 (EVS steps 1-4, eq. 4.1-4.4; App. 2 splitting identities).
* ``vtm``      — §5 (eq. 5.6-5.8 and Table 1): local SPD systems, the (u, omega) iteration,
                 assembly of the solution, FP64 residual, direct solve.
* ``matching`` — §7.1 (Def. 7.1 input impedance, impedance matching).
* ``theory``   — App. 3 (the port-space iteration operator of eq. A3.8) and the closed-form
                 reflection of a single transmission line (§2 eq. 2.1 with §7.1).
* ``mixed``    — Table 1 with reduced-precision local factors inside FP64 defect correction
                 (error statements for the FP32 / FP16 paths).
* ``coupled``  — §7.2 and Thm 7.1: coupled lines (bundle admittance matrices), the multi-conductor
                 reflection law, candidate line pairs.
* ``conformal``— App. 1 and Thm 4.2: the general conformal split of an SPD matrix by completing the
                 square over each interior.
* ``n2n``      — Table 1 as neighbour-to-neighbour message passing, one thread per subgraph, with
                 late, reordered and dropped messages (host-side failure detection).
* ``mlp``, ``features`` — the FP64 perceptron and line features the learned impedances are
                 checked against.

Pins (what fixes each function independently of itself) are listed in each module header.
"""
