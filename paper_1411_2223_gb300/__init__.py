"""GB300-native asqtad staggered CG (mixed-precision CG inverter on
m^2 - D_eo D_oe with a hand-written sm_103a Dslash), behind the C ABI of
include/sq.h.  ``paper_1411_2223_gb300.sq`` is the Python binding and
``paper_1411_2223_gb300.build`` compiles the library."""
