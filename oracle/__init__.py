"""CPU oracles for the reproducible grouped SUM (TEST INFRASTRUCTURE ONLY).

``exact``  -- Python big-integer model (definition form + Algorithm 2 replay).
``oracle`` -- ctypes binding of ``repro_oracle.c`` (Algorithm 2 in IEEE
              arithmetic, the paper's <S, C> state).

Only tests/, __graft_entry__.smoke() and bench.py's CPU-baseline leg may use
this package; the library's CUDA path must never import it.
"""
