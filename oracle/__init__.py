"""FP64 CPU oracle of the data-driven (DD) projection hot path.

TEST INFRASTRUCTURE ONLY.  Nothing in the product package imports, links or
executes this package; it is used by ``tests/``, by ``__graft_entry__.smoke()``
(to check one small GPU invocation) and by the CPU-baseline leg of
``bench.py``.  It shares no code with the CUDA path: only the seeded input
generators of ``dd_inputs`` feed both.

Contents, each following the paper (Eggersmann, Stainier, Ortiz & Reese,
"Efficient Data Structures for Model-free Data-Driven Computational
Mechanics", arXiv:2012.00357):

* ``metric``  - the local distance of Eq. (3) and the Euclidean map
                 q = (C^{1/2} eps, C^{-1/2} sig) of Sec. 3.2, scaled by 1/sqrt(2)
                 so that |dq|^2 carries the 1/2 of Eq. (2).
* ``nn``      - exact nearest-neighbour projection P_D, Eq. (7), as a plain
                 brute-force scan in C (the linear search of Sec. 1).
* ``fem``     - trilinear hexahedral finite elements, the operators of
                 Eq. (5)-(6), direct sparse LU of the fixed stiffness (Sec. 2).
* ``dd``      - the fixed-point iteration z_{i+1} = P_D(P_C(z_i)), Eq. (8).
* ``ann``     - the approximate, warm-started k-means-partition search
                 rules of Sec. 4.2-4.5 (Eq. 13, Eq. 14).
"""
